/*
 * psp.h -- C ABI of libpsp, a GB300 (sm_103a) implementation of PSP-GMRES
 * (Ghasemi & Taylor, "A Progressive Statistical Method for Preconditioning Matrix-Free
 * Solution of High-Order Discretization of Linear Time-Dependent Problems",
 * arXiv:1308.5626).
 *
 * One call of psp_step solves the implicit-Euler system of Eq. 4,
 *     A u^{n+1} = u^n,   A = I - dt L,
 * where L is the high-order finite-difference operator of Eqs. 1-2 on a periodic grid,
 * by the restarted, right-preconditioned, matrix-free GMRES of Algorithm 1.  Every
 * matvec pair (x, A x) is kept as a history; after the step the banded preconditioner N
 * is fitted to that history row by row (Algorithm 2, MREP) and preconditions the next
 * step.
 *
 * Conventions shared by every entry point:
 *  - Vectors are flattened grids with x fastest (index = ix + nx*(iy + ny*iz)).
 *  - Pointers named *_host are host memory; every other array pointer is DEVICE memory
 *    owned by the caller (e.g. a torch tensor's data_ptr).  The library never frees
 *    caller memory and keeps no pointer to it after the call returns.
 *  - Band storage of an n x n banded matrix with half-width b is row-major
 *    n x (2b+1) doubles: band[i*(2b+1) + p] = N(i, i + p - b).  Entries whose column
 *    falls outside [0, n) are ignored on input and written as 0 on output.
 *  - The library owns its workspace (Krylov basis, history ring, Hessenberg data, band
 *    factors) and allocates it when the handle is created.  Some calls allocate more on
 *    their first use and keep it: psp_step_host and the integrators (two n-vectors each),
 *    and psp_step_batch (its batched-launch buffers and its host threads' streams);
 *    psp_fit_band_static allocates nothing.
 *  - All device work is enqueued on the stream given to psp_create, except on
 *    psp_step_batch's graph path, which steps a handle on a stream of the library that is
 *    joined to the handle's stream by events at both ends of the call.  psp_step,
 *    psp_fit_band*, psp_set_band and psp_step_host synchronise that stream before they
 *    return; the other calls are asynchronous.
 *  - The host-side phases (psp_step, each segment of restart cycles, the fit, the batch
 *    calls, psp_step_host) are marked by NVTX ranges for timeline tools.
 *  - No exception crosses the ABI.  A failing call returns a status other than PSP_OK
 *    and leaves a thread-local message for psp_last_error().
 *  - A handle must not be used by two host threads at once.
 */
#ifndef PSP_H
#define PSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psp_ctx *psp_handle;

typedef enum {
  PSP_OK = 0,
  PSP_ERR_ARG = 1,     /* invalid argument; nothing was enqueued */
  PSP_ERR_CUDA = 2,    /* a CUDA runtime call failed */
  PSP_ERR_OOM = 3,     /* device allocation failed (psp_create only) */
  PSP_ERR_NOCONV = 4,  /* max_restarts reached; the output holds the last iterate */
  PSP_ERR_NUMERIC = 5, /* NaN/Inf in a residual norm, or a singular band factor */
  PSP_ERR_DEVICE = 6   /* the device reported an internal error flag */
} psp_status;

enum { PSP_FP64 = 0, PSP_MIXED = 1 };

/* psp_step_info.flags bits */
#define PSP_FLAG_SINGULAR_FIT 0x1       /* the last fit had degenerate rows (identity rows written) */
#define PSP_FLAG_CANDIDATE_TRIED 0x2    /* this step tried a freshly fitted N on its first cycle */
#define PSP_FLAG_CANDIDATE_ACCEPTED 0x4 /* ... and adopted it */
#define PSP_FLAG_FACTOR_FAILED 0x8      /* a fitted N had a zero pivot and was dropped */
#define PSP_FLAG_BREAKDOWN 0x10         /* an Arnoldi breakdown ended a cycle */
#define PSP_FLAG_FITTED 0x20            /* Algorithm 2 fitted a candidate N after this step */
#define PSP_FLAG_DF_RESTART 0x40        /* mixed form: a cycle's restart residual r = B - A X_0 was
                                           computed in double-float FP32 pairs (about 48 bits;
                                           taken when tol >= 2^-42 sum|coefficients of A|) */

/* Periodic grid of Eq. 1: ndim in {1,2,3}, n[d] points on [0, length[d]), h = length/n. */
typedef struct {
  int ndim;
  int64_t n[3];
  double length[3];
} psp_grid;

/* One term alpha * d^k u / dx_dir^k of the operator L (Eq. 1); k in 1..4. */
typedef struct {
  int k;
  int dir;
  double alpha;
} psp_term;

#define PSP_SOLVER_GMRES 0
#define PSP_SOLVER_BICGSTAB 1

typedef struct {
  int precision;     /* PSP_FP64 (default): every vector in FP64.  PSP_MIXED: Krylov
                        vectors, history, stencil and band solve in FP32 with FP32
                        accumulation; Hessenberg/Givens, band fit and the per-restart true
                        residual and solution update in FP64. */
  int intercept;     /* 1 (default): Algorithm 2's design row of ones; 0: without it */
  int max_restarts;  /* n_r of Algorithm 1 (default 200) */
  int max_hist_cols; /* history ring length M_max (default 2(m+1)) */
  double inner_tol;  /* PSP_MIXED: a cycle ends once R(k) <= inner_tol * ||r_restart||
                        (default 1e-5); the step ends on the FP64 true residual */
  int accept_rule;   /* 1 (default): a fitted N is adopted only if it converges at least
                        as fast on the next step's first cycle; 0: always adopt */
  int fuse_matvec;   /* 1 (default): the Arnoldi matvec w = A N^{-1} v runs inside the first
                        Gram-Schmidt pass when every grid row is a whole number of 16-byte
                        vectors wider than the stencil halo; 0: as a kernel of its own.
                        Same arithmetic either way. */
  int adjoint;       /* 0 (default): the handle solves with A = I - dt L.  1: with
                        A^T = I - dt L^T (every stencil mirrored, w_j -> w_-j, exact on the
                        periodic grid): the adjoint system of a step, for gradients. */
  int cyclic;        /* 0 (default): Algorithm 2's boundary rows (the first and last b rows
                        of N keep only N(i,i), from a simple linear fit).  1: cyclic band for a
                        periodic 1D grid (psp_create with ndim = 1 and n >= 4b+2, else
                        PSP_ERR_ARG): every row regresses on rows i-b..i+b modulo n, and the
                        band storage reads band[i][p] = N(i, (i+p-b) mod n) everywhere (fit,
                        psp_set_band, psp_get_band, the solves).  The solve treats the
                        wrapped corner entries exactly (Sherman-Morrison-Woodbury on the
                        in-range band; a singular capacitance matrix drops the N like a zero
                        pivot).  Not in the paper; for a periodic 1D stencil N = A can then be
                        fitted exactly. */
  int solver;        /* PSP_SOLVER_GMRES (default): Algorithm 1.  PSP_SOLVER_BICGSTAB:
                        restarted right-preconditioned BiCGSTAB (van der Vorst 1992), m
                        iterations per restart cycle, each storing its two matvec pairs
                        (p^, A p^), (s^, A s^) -- scaled by 1/||r|| -- in the same history, so
                        the fit, the acceptance rule and the preconditioner are unchanged.
                        PSP_FP64 and m >= 3 only (else PSP_ERR_ARG); the profiling mode
                        times GMRES cycles only.  Not in the paper. */
  int onchip;        /* -1 (default): the on-chip path for systems of at most 32768 unknowns;
                        1: for systems of at most 262144 unknowns; 0: never.  On the on-chip
                        path one CTA runs every restart cycle of a step (restart, band solve,
                        matvec, Gram-Schmidt, Givens, update) with the cycle loop on the device,
                        so the host waits once per step instead of once per cycle, and
                        psp_step_batch runs all its handles' cycles in shared launches (one
                        CTA per system).  Its Gram-Schmidt is classical applied twice (CGS2).
                        GMRES only (BiCGSTAB handles take the cycle graphs); the profiling mode
                        does not time it. */
  int cycle_loop;    /* 1: on the captured-graph path the restart loop runs on the
                        device -- one graph launch runs cycle after cycle (a CUDA graph WHILE
                        node) until the step converges, a cycle breaks or the segment's cycle
                        budget is spent, and the host waits once per segment (the acceptance
                        rule's trial cycle is a segment of one cycle).  0 (default): one graph
                        launch and one host round trip per restart cycle.  Same iterates either
                        way; the profiling mode runs per cycle.  Falls back to 0 if the runtime
                        refuses the conditional graph.  Measured: no change on a 256^3 step,
                        0.5% faster at 1024^2 (30 cycles per step), 22-25% slower aggregate
                        for 512 concurrent small instances (psp_step_batch). */
} psp_opts;

typedef struct {
  int iters;         /* Arnoldi iterations (preconditioned matvecs) of the step */
  int cycles;        /* restart cycles */
  int status;        /* psp_status of the step */
  int flags;         /* PSP_FLAG_* */
  double rel_res;    /* PSP_FP64: Givens estimate R(k)/||u^n|| at exit;
                        PSP_MIXED: FP64 true residual ||u^n - A u^{n+1}|| / ||u^n|| */
  int hist_cols;     /* valid history columns after the step */
  int singular_rows; /* degenerate rows in the fit made after the step (0 if no fit was
                        made: none is made while the acceptance rule's back-off keeps
                        the next step from trying a candidate) */
  int launches;      /* CUDA kernels this step launched (every kernel node of every
                        replayed cycle graph, plus the fit and factorisation kernels) */
} psp_step_info;

/* Kernel classes timed by the profiling mode (psp_set_profiling). */
enum {
  PSP_K_PRECOND = 0, /* preconditioner solve Y_k = N^{-1} V(:,k) (all its kernels) */
  PSP_K_STENCIL = 1, /* matvec U_k = A Y_k */
  PSP_K_CGS1 = 2,    /* orthogonalisation pass A: block dot products [V, v_j]^T [v_j, w_j] */
  PSP_K_CGS2 = 3,    /* (unused: the orthogonalisation needs two passes) */
  PSP_K_CGS3 = 4,    /* pass B: q_j, v_{j+1}, completed Hessenberg column, Givens, finish test */
  PSP_K_COUNT = 5
};

typedef struct {
  double ms[PSP_K_COUNT];    /* summed device time per kernel class */
  double bytes[PSP_K_COUNT]; /* summed algorithmic bytes per kernel class */
  int64_t launches[PSP_K_COUNT]; /* timed launches per kernel class */
} psp_profile;

/* Fill *opts with the defaults listed above.  Returns PSP_ERR_ARG for NULL. */
psp_status psp_default_opts(psp_opts *opts);

/*
 * Create a solver for A = I - dt L on `grid`, L = sum over `terms` of
 * alpha * h^-k * (central difference of accuracy `order`) (Eqs. 1-2; order in
 * {2,4,6,8}), band half-width b in 1..4 (the paper's d of Algorithm 2), restart length
 * m in 1..64 (n_A of Algorithm 1).  `opts` may be NULL (defaults).  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  Every direction needs n[d] >= 2r+1 for
 * the widest stencil radius r and the grid needs at least 2b+1 points.  Allocates all
 * workspace on the current device; PSP_ERR_OOM if it does not fit.
 */
psp_status psp_create(const psp_grid *grid, int order, const psp_term *terms, int nterms,
                      int b, int m, const psp_opts *opts, void *cuda_stream, psp_handle *out);

/*
 * A handle whose operator is an explicit banded matrix instead of the stencil: the paper's
 * mock test (Results section: a random seven-diagonal A, diagonally dominant, u^n = 1..n).
 * A_band is a device array of n x (2w+1) doubles, row-major band storage
 * A(i, i+p-w) = A_band[i (2w+1) + p] (entries outside the matrix ignored), copied into the
 * handle (FP64 and FP32).  psp_step then solves A u_np1 = u_n (dt is ignored) with the same
 * restarted PSP-GMRES, history and band fit of half-width b; psp_matvec applies A, and with
 * opts->adjoint A^T.  psp_apply_L returns PSP_ERR_ARG (there is no L).  w in 1..64.
 */
psp_status psp_create_banded(int64_t n, const double *A_band, int w, int b, int m, const psp_opts *opts,
                             void *cuda_stream, psp_handle *out);

/* Release every resource of the handle.  NULL is accepted. */
psp_status psp_destroy(psp_handle h);

/* Message of the last failing call on this host thread ("" if none). */
const char *psp_last_error(void);

/*
 * One implicit-Euler step (Eq. 4): u_np1 = A^{-1} u_n to the relative tolerance tol
 * (||u_n - A u_np1|| <= tol ||u_n||), by Algorithm 1 with X_0 = u_n, B = u_n and the
 * adopted preconditioner N (identity until a fit was adopted), followed by the
 * Algorithm 2 fit of a candidate N for the next step (not made while the acceptance
 * rule's back-off keeps the next step from trying a candidate).  u_n and u_np1 are device arrays
 * of n doubles and must not overlap.  `info` (host) may be NULL.  The history persists
 * across steps while dt is unchanged and is cleared when dt changes.  The work runs on the
 * handle's stream and u_np1 is complete when the call returns.
 * Returns PSP_ERR_NOCONV after max_restarts cycles (u_np1 = last iterate).
 */
psp_status psp_step(psp_handle h, const double *u_n, double *u_np1, double dt, double tol,
                    psp_step_info *info);

/*
 * One implicit step of many independent handles (a batch of independent systems, e.g.
 * 512 1D and 2D grids of 2^10 to 2^18 points): handle i steps u_n[i] -> u_np1[i] with dt[i] and the common tolerance
 * tol, exactly as psp_step would.  The handles on the on-chip path (opts.onchip; those of the
 * first one's precision) run the restart cycles of all their steps in shared persistent
 * launches, one CTA per system taken from a work counter, largest first, one launch per CTA
 * size and per round of the acceptance rule's decisions; the other handles are stepped
 * concurrently by nthreads host threads, each stepping one handle at a time on a stream of its
 * own (created by the library on first use and kept), so up to nthreads instances' cycle
 * graphs run on the GPU concurrently even where handles share a stream.  A handle's work in
 * the call follows the work already enqueued on its stream, and work enqueued on that stream
 * later follows it (event joins at both ends).  The batched launches take device and
 * pinned buffers made on the first such call (and grown for a larger batch).  infos, seconds
 * and statuses are host arrays of count entries or NULL; seconds is each instance's time:
 * host wall time of its step on the graph path, device time of its cycles (the GPU clock) plus
 * host time of its fit on the on-chip path.  Returns PSP_OK, PSP_ERR_NOCONV if an instance
 * reached max_restarts, or the first other error status of an instance (all instances are
 * attempted).  A handle must not appear twice.  See psp_batch_tuner.
 */
psp_status psp_step_batch(psp_handle *handles, int count, const double *const *u_n, double *const *u_np1,
                          const double *dt, double tol, int nthreads, psp_step_info *infos, double *seconds,
                          psp_status *statuses);

/* The batch autotuner of psp_step_batch (not in the paper).  mode 1 switches it on and
 * forgets what it measured, 0 switches it off (the handles keep the execution it last gave
 * them), -1 only reports.  While on, psp_step_batch runs every instance of a size class
 * (floor(log2 n)) the same way on a call: through the captured cycle graphs, or (for classes
 * up to 2^16 unknowns) on the on-chip path with CTAs of 128, 256 or 512 threads -- one
 * candidate per call until each was
 * measured, then the one whose calls took the least wall time per Arnoldi iteration of the
 * whole batch (the classes share the GPU, so the call's time, not an instance's own, is what an
 * execution costs the batch), and it sets the handles' opts.onchip and CTA size accordingly
 * (later psp_step calls on them run the same way).
 * classes (host, max_classes entries, may be NULL) receives one entry per size class seen;
 * *nclasses (may be NULL) their number. */
typedef struct {
  int log2_n;            /* size class: floor(log2 n) */
  int choice;            /* -1: not decided; 0: cycle graphs; 128, 256, 512: on-chip CTA size */
  int samples[4];        /* measured calls: graphs, on-chip 128, 256, 512 */
  double us_per_iter[4]; /* wall time of those calls per Arnoldi iteration of the batch (microseconds) */
} psp_tuning_class;
psp_status psp_batch_tuner(int mode, psp_tuning_class *classes, int max_classes, int *nclasses);

/* Second-order implicit integrators on the step (not in the paper): each solves with the
 * same matrix-free PSP-GMRES and progressive preconditioner as psp_step, on another
 * right-hand side and a scaled time step.  Vectors are device FP64 arrays of n values (u_np1
 * must not overlap the inputs); info sums iterations, cycles and launches over the solves.
 * PDE handles only (psp_create; PSP_ERR_ARG for psp_create_banded handles).
 *
 * psp_step_bdf2: BDF2, (I - 2/3 dt L) u^{n+1} = (4 u^n - u^{n-1}) / 3 -- one step of the
 *   handle at dt' = 2 dt / 3 (start a BDF2 run with one psp_step for u^1).
 * psp_step_sdirk2: Alexander's two-stage L-stable SDIRK (gamma = 1 - 1/sqrt 2):
 *   (I - gamma dt L) U1 = u^n; (I - gamma dt L) u^{n+1} = u^n + (1 - gamma) dt L U1 --
 *   two steps of the handle at gamma dt, so both stages share the history and N.
 *   A stage that reaches max_restarts gives PSP_ERR_NOCONV after the second stage ran. */
psp_status psp_step_bdf2(psp_handle h, const double *u_nm1, const double *u_n, double *u_np1, double dt,
                         double tol, psp_step_info *info);
psp_status psp_step_sdirk2(psp_handle h, const double *u_n, double *u_np1, double dt, double tol,
                           psp_step_info *info);

/* psp_step on host arrays: copies u_n_host to the device, steps, copies the result to
 * u_np1_host (both n doubles, pageable or pinned). */
psp_status psp_step_host(psp_handle h, const double *u_n_host, double *u_np1_host, double dt,
                         double tol, psp_step_info *info);

/* y = A x = x - dt L x (the matrix-free product of Algorithm 1), FP64 / FP32 device
 * arrays of n elements; x and y must not overlap. */
psp_status psp_matvec(psp_handle h, const double *x, double *y, double dt);
psp_status psp_matvec_f32(psp_handle h, const float *x, float *y, double dt);

/*
 * Algorithm 2 (MREP) on a caller-given history: Px, Py are n x M column-major device
 * arrays (column c starts at c*ld, ld >= n), N_band is the device output (band storage,
 * half-width b of the handle).  Rows 0..b-1 and n-b..n-1 get the slope of a simple
 * linear fit on the diagonal; interior rows the least-squares fit on
 * [1; Px(i-b..i+b, :)] (or without the row of ones when opts.intercept = 0).  With
 * opts.cyclic every row is an interior row, its neighbours taken modulo n.  Rows whose
 * normal equations are degenerate (relative Cholesky pivot <= 1e-12) get the identity
 * row; their count goes to *singular_rows (host, may be NULL).  Requires M >= 1.
 * Does not change the handle's preconditioner.
 */
psp_status psp_fit_band(psp_handle h, const double *Px, const double *Py, int64_t ld, int M,
                        double *N_band, int *singular_rows);
psp_status psp_fit_band_f32(psp_handle h, const float *Px, const float *Py, int64_t ld, int M,
                            double *N_band, int *singular_rows);

/*
 * Allocation-free band fit (the paper has no counterpart: this is a deployment variant of
 * psp_fit_band above).  For callers that cannot allocate device memory -- e.g. code in an
 * allocation-free real-time or graph-driven loop, or a plugin given a fixed memory budget --
 * and so cannot create a handle (psp_create allocates the solver workspace).  Same result
 * as psp_fit_band for a handle with half-width b, the given intercept flag and
 * opts.cyclic = 0: the first and last b rows are Algorithm 2's boundary rows (there is no
 * cyclic variant).  Px, Py are n x M column-major FP64 device arrays (leading dimension
 * ld >= n), N_band the device output (n x (2b+1) band storage), *singular_rows (host, may be
 * NULL) the count of degenerate rows.  Work is enqueued on cuda_stream (a cudaStream_t,
 * NULL = legacy default) and the call returns after it finished if singular_rows is not
 * NULL; singular_rows must be NULL while cuda_stream is being captured into a graph
 * (PSP_ERR_ARG otherwise), because reading the count back synchronises the stream.
 * Scratch: a static device array for at most 65536 rows (10 MiB per GPU that loads the
 * library, kept until exit); larger n returns PSP_ERR_ARG.  The first call on a device
 * looks up that array's device address (do it before any stream capture).  All calls share
 * the array: calls that overlap on the GPU race and must be serialised by the caller.
 */
psp_status psp_fit_band_static(const double *Px, const double *Py, int64_t ld, int M, int64_t n, int b,
                               int intercept, double *N_band, int *singular_rows, void *cuda_stream);

/*
 * The matvec history of Algorithm 1 that the next Algorithm 2 fit would use: the valid
 * columns of the handle's history ring (at most max_hist_cols, the most recent pairs
 * (x, A x) of the steps since the history was last cleared), oldest first, copied to Px, Py
 * as n x cols column-major FP64 device arrays with leading dimension ld >= n (FP32 history of
 * the mixed form widened exactly).  *cols (host) receives the number of valid columns; with
 * Px or Py NULL only that count is returned.  PSP_ERR_ARG if max_cols is smaller than it.
 * Synchronous.  Diagnostics and checkpoints: with psp_get_band it is the state that
 * decides the next step's preconditioner.
 */
psp_status psp_get_history(psp_handle h, double *Px, double *Py, int64_t ld, int max_cols, int *cols);

/* Factor the device band N_band (half-width b) and adopt it as the preconditioner.
 * Returns PSP_ERR_NUMERIC (and keeps the previous N) if a pivot of the partitioned
 * factorisation is zero or not finite. */
psp_status psp_set_band(psp_handle h, const double *N_band);

/* Copy the adopted N to the device array N_band (identity band if none is adopted). */
psp_status psp_get_band(psp_handle h, double *N_band);

/* y = N^{-1} v with the adopted N (the preconditioner solve of Algorithm 1), or
 * y = N^{-T} v with transpose = 1 (the preconditioner of the adjoint system); device
 * arrays of n elements; v and y may be the same array.  The first transposed solve after
 * the adopted N changed factors N^T (synchronous); PSP_ERR_NUMERIC if that fails.  With
 * no adopted N both are copies (N = I). */
psp_status psp_apply_precond(psp_handle h, const double *v, double *y, int transpose);
psp_status psp_apply_precond_f32(psp_handle h, const float *v, float *y, int transpose);

/* y = L x (term < 0) or y = D_t x (0 <= term < nterms: term t of psp_create with unit
 * alpha, i.e. h^-k times the central difference of order k along its direction), FP64
 * device arrays of n elements that must not overlap.  On an adjoint handle L^T and D_t^T.
 * With u^{n+1} = A^{-1} u^n, A = I - dt L, L = sum_t alpha_t D_t and an adjoint state
 * lambda = A^{-T} g, the gradients of a loss with dL/du^{n+1} = g are lambda (u^n),
 * lambda . L u^{n+1} (dt) and dt lambda . D_t u^{n+1} (alpha_t).  Synchronous. */
psp_status psp_apply_L(psp_handle h, int term, const double *x, double *y);

/* The gradients of a loss through one implicit step with respect to dt and the term
 * coefficients, from the adjoint state (derivative of Eq. 4, not in the paper): with
 * u = u^{n+1} = A^{-1} u^n, A = I - dt L, L = sum_t alpha_t D_t and lambda = A^{-T} g for
 * g = dLoss/du^{n+1},
 *     grads_host[0]     = dLoss/d dt      = lambda . L u = sum_t alpha_t (lambda . D_t u),
 *     grads_host[1 + t] = dLoss/d alpha_t = dt (lambda . D_t u),   t < nterms of psp_create.
 * lam and u are FP64 device arrays of n values; the dot products are made by one kernel per
 * 16 terms with a fixed-order reduction (deterministic).  Forward PDE handles only
 * (PSP_ERR_ARG for an adjoint or banded handle).  Synchronous. */
psp_status psp_adjoint_grads(psp_handle h, const double *lam, const double *u, double dt, double *grads_host);

/* Adopt the preconditioner of handle src (its adopted N, or I if it has none) in handle dst,
 * transposed (N^T) with transpose = 1: the adjoint system A^T lambda = g is preconditioned by
 * N^T of the forward handle's N.  Both handles need the same n, b and cyclic option, on the
 * current device.  dst's own candidate and history are kept.  PSP_ERR_NUMERIC (dst keeps its
 * N) if the factorisation fails.  Synchronous. */
psp_status psp_set_band_from(psp_handle dst, psp_handle src, int transpose);

/* Stencil of L without dt: w_host[d*(2R+1) + (j+R)] is the weight of u(x + j h e_d) in
 * (L u)(x) for d < ndim and j in -R..R, R = *radius (host).  w_host holds 3*(2R+1)
 * doubles; pass NULL to query only the radius. */
psp_status psp_get_stencil(psp_handle h, double *w_host, int *radius);

/* Forget the adopted N, the candidate and the history (back to N = I). */
psp_status psp_reset(psp_handle h);

/* Profiling mode (off by default).  When on, the captured restart cycles carry CUDA
 * event records around every kernel class of every fourth Arnoldi iteration (k = 1, 5,
 * 9, ...), and psp_step adds the device time of those that ran (k <= k_end) to a running
 * psp_profile,
 * together with each launch's algorithmic bytes (the reads and writes the operation needs
 * at least once: (j+3) s n for pass A with the matvec folded in, (j+4) s n for pass B,
 * (2b+3) s n for a band solve, s the element size).  psp_get_profile copies the running totals to
 * *out (host) and, if reset != 0, zeroes them. */
psp_status psp_set_profiling(psp_handle h, int enable);

/* Diagnostics: the Givens residuals R(1..k_end) of the last restart cycle of the last
 * psp_step (Algorithm 1), at most maxk of them, to R_host; *k_end (host) = k_end. */
psp_status psp_last_cycle_residuals(psp_handle h, double *R_host, int maxk, int *k_end);
psp_status psp_get_profile(psp_handle h, psp_profile *out, int reset);

#ifdef __cplusplus
}
#endif
#endif /* PSP_H */
