/*
 * superscs.h -- C ABI of the GB300-native SuperSCS solver (libsuperscs.so).
 *
 * Method: Sopasakis, Menounou, Patrinos, "SuperSCS: fast and accurate
 * large-scale conic optimization", arXiv 1903.06477.
 *
 * Problem (Sec. 3, primal (P)):   minimize <c,x>  s.t.  b - A x = s,  s in K
 * Dual    (Sec. 3, (D)):          minimize <b,y>  s.t.  y in K*,  A^T y + c = 0
 * The solver applies Douglas-Rachford splitting to the homogeneous self-dual
 * embedding (Sec. 3.1, Eq. drs) and globalises it with SuperMann
 * (Algorithm 1) using restarted Broyden (Algorithm 2) or Anderson directions
 * (Sec. 4.4).  Every step runs in hand-written CUDA kernels for sm_103a.
 *
 * Conventions
 *  - Cone rows of s are ordered [ f zero | l orthant | q SOCs | s PSDs |
 *    ep primal exponential cones | ed dual exponential cones ].
 *    An SOC block (x, t) stores t LAST (Sec. 2, cone (iii)).  A PSD block of
 *    order d occupies d(d+1)/2 rows holding svec(X): lower triangle, column
 *    by column, off-diagonal entries multiplied by sqrt(2) (Sec. 2, map mat).
 *  - A is CSR with m rows: Ap[m+1] (int64, Ap[0] = 0), Ai[nnz] (int32 column
 *    indices in [0,n)), Ax[nnz].  nnz must be below 2^31.
 *  - HSDE vectors u = (chi, psi, tau) have N = n + m + 1 entries (Sec. 3.1).
 *  - All input arrays are caller-owned and only read.  scs_setup copies them
 *    to the device.  Output and vector arguments may be host or device
 *    pointers (unified addressing decides the copy direction).
 *  - Every function returns SCS_OK (0) or a negative error code and never
 *    aborts; the algorithmic outcome is reported in scs_info.status.
 */
#ifndef SUPERSCS_H
#define SUPERSCS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define SCS_OK 0
#define SCS_EINVAL (-1)   /* bad sizes, cone dims not summing to m, non-finite data, bad settings */
#define SCS_ENOMEM (-2)   /* device or host allocation failed */
#define SCS_ECUDA (-3)    /* a CUDA call failed; see scs_last_error */
#define SCS_ETIMEOUT (-4) /* a device-wide barrier waited more than 10 s; the solve was abandoned */

/* scs_info.status (Sec. 3.1 recovery rules and Sec. 4.3 certificates) */
#define SCS_SOLVED 1
#define SCS_INFEASIBLE (-1)
#define SCS_UNBOUNDED (-2)
#define SCS_MAX_ITERS (-3)
#define SCS_TIME_LIMIT (-4)
#define SCS_NUMERICAL (-5)

/* directions (Sec. 4.4) */
#define SCS_DIR_AA 0   /* Anderson's acceleration */
#define SCS_DIR_RB 1   /* restarted Broyden, Algorithm 2 */
#define SCS_DIR_NONE 2 /* d = 0: with c0 = 0 every step is the KM step of Eq. (km) */
#define SCS_DIR_AA_QR 3 /* Anderson's acceleration with its least squares solved through a QR
                           factorisation of the window, updated as pairs enter (Gram-Schmidt)
                           and leave (Givens rotations), Sec. 4.4 */

/* precision */
#define SCS_FP64 0  /* every vector and the matrix in FP64 */
#define SCS_MIXED 1 /* FP32 bulk (matrix, vectors, CG, projections), FP64 scalars and
                       reductions, then an FP64 refinement phase that confirms eps */

/* execution team */
#define SCS_TEAM_AUTO 0
#define SCS_TEAM_BLOCK 1 /* one thread block per instance */
#define SCS_TEAM_GRID 2  /* every SM on one instance (cooperative launch) */

typedef struct {
    int32_t f, l;        /* zero-cone rows, orthant rows (Sec. 2 cones (i), (iv)) */
    int32_t nq;          /* number of SOCs */
    const int32_t *q;    /* SOC dimensions, each >= 1 (Sec. 2 cone (iii)) */
    int32_t ns;          /* number of PSD blocks */
    const int32_t *s;    /* PSD orders d, each 1..1024 (Sec. 2 cone (ii)); blocks up to 64 are
                            decomposed in shared memory, larger ones in a global-memory workspace
                            of about 2 d^2 words (plus d^2 doubles for SCS_MIXED) per block */
    int32_t ep;          /* primal exponential cones (Sec. 2 cone (v)), 3 rows each:
                            (x1, x2, x3) with x1 >= x2 exp(x3 / x2), x2 > 0, closure */
    int32_t ed;          /* dual exponential cones, 3 rows each: (y1, y2, y3) with
                            -y3 exp(y2 / y3) <= e y1, y3 < 0, closure */
} scs_cone;

typedef struct {
    int32_t m, n;
    const int64_t *Ap;
    const int32_t *Ai;
    const double *Ax;
    const double *b; /* m */
    const double *c; /* n */
} scs_data;

typedef struct {
    int32_t direction;   /* SCS_DIR_AA | SCS_DIR_RB | SCS_DIR_NONE | SCS_DIR_AA_QR */
    int32_t mem;         /* memory of the direction (AA, AA_QR: 1..32, RB: 0..64) */
    double eps;          /* tolerance of Sec. 4.3 on pr, dr, gap, ic, uc */
    double c0, c1, q, sigma, lambda; /* Algorithm 1 parameters */
    double thetabar;     /* Powell safeguard of Algorithm 2 */
    int32_t max_iters;   /* outer iterations of Algorithm 1 */
    int32_t ls_max;      /* backtracking halvings before the KM fallback (alpha = 0) */
    int32_t cg_max;      /* CG iterations per linear solve */
    int32_t check_every; /* termination test period */
    double cg_rtol;      /* CG stops when ||res|| <= cg_rtol ||rhs|| */
    double time_limit_s; /* <= 0: none */
    int32_t precision;   /* SCS_FP64 | SCS_MIXED */
    int32_t warm;        /* 0: u0 = (0,0,1);  1: u0 = warm_u */
    const double *warm_u;/* N values (host or device) when warm = 1 */
    int32_t verbose;
    double aa_reg;       /* Tikhonov factor of the AA normal equations */
    int32_t team;        /* SCS_TEAM_* */
    int32_t threads;     /* threads per block, 0 = automatic (grid team: 512, its maximum;
                            block team: 256, or the batch autotuner's choice) */
    double mixed_cg_rtol;   /* CG tolerance of the FP32 phase (SCS_MIXED) */
    int32_t mixed_stall;    /* FP32 phase ends after this many iterations without a
                               10% drop of ||Ru|| below its best value (SCS_MIXED) */
    int32_t mixed_max_iters;/* cap on FP32-phase iterations (SCS_MIXED) */
    double mixed_switch;    /* FP32 phase hands over to FP64 once max(pr,dr,gap) <= this (SCS_MIXED) */
    double cg_adapt;        /* > 0: inside the loop CG also stops at ||res|| <= cg_adapt ||Ru||
                               (not in the paper; 0 keeps the fixed relative tolerance) */
    int32_t spmv_path;      /* sparse products of the grid team.  0: automatic -- the column-blocked
                               layout (each CTA's rows against every column block, vector slices
                               staged in shared memory per block, one CTA per SM) where each (CTA,
                               column block) holds at least 1024 entries on average, else sliced
                               ELL; 1: sliced ELL, direct streaming loads; 2: sliced ELL, TMA-staged
                               stream; 3: column-blocked wherever the layout fits shared memory;
                               4: two-dimensional tiles (one row block x column block per CTA, the
                               vector's column block resident in shared memory, partial sums added
                               by a second pass) wherever a split fits, else as 3.  The tiles
                               measured 10-15% slower than the column-blocked layout on the 1e7-
                               nonzero benchmark matrix, so the automatic rule does not take them.
                               The block team always uses sliced ELL. */
    int32_t warm_fallback;  /* > 0: a warm start whose ||Ru|| is not below the cold start's ||Ru0||
                               after this many iterations is abandoned for the cold start */
    int32_t mixed_resume;   /* SCS_MIXED, 1 (default): the FP64 phase continues Algorithm 1 from the
                               FP32 phase's state -- its direction memory (AA pairs and Gram matrix,
                               or the Broyden pairs), the pending secant pair, eta, eta0, r_safe and
                               the outer index of q^nu; 0: it restarts Algorithm 1 from the FP32
                               iterate */
    int32_t mixed_refine;   /* SCS_MIXED, 1 (default): the FP64 phase solves each linear system of
                               Sec. 4.1 by iterative refinement -- residuals with the FP64 matrix,
                               corrections by CG with the FP32 copy -- so its FP64 work is a few
                               sparse products per solve; 0: plain FP64 CG */
    int32_t linsys_direct;  /* 1: instances run by one thread block (the block team, every batch
                               instance) with n <= 4096 form I + A^T A densely at setup, factor it
                               L L^T in each precision (the "direct" solve Sec. 4.1 names beside CG)
                               and solve each linear system by two blocked triangular solves; the
                               factor takes n^2 words per precision.  0 (default): CG.  Ignored by
                               the grid team.  A non-positive pivot makes setup fail with SCS_EINVAL */
    int32_t mixed_stall_after_tau; /* SCS_MIXED, 1 (default): while the FP32 phase's termination test
                               sees tau_ = 0, or max(pr, dr, gap) above 100 mixed_switch, its stall
                               window is 5 mixed_stall iterations -- the residuals of Sec. 4.3 are
                               undefined with tau_ = 0 and ||Ru|| may plateau while the iterate turns
                               away from the tau axis, and a plateau that far above the hand-over
                               level is a pause of Algorithm 1, not the FP32 floor; 0: mixed_stall
                               throughout */
    double psd_recheck_tol; /* SCS_MIXED with PSD cones: every FP32 eigendecomposition of a PSD block
                               (Sec. 2, cone (ii)) is checked in FP64, ||X V - V L||_F / ||X||_F; a
                               block above this bound is decomposed again in FP64 and projected from
                               that.  Default 1e-4, ten times the largest residual of converged FP32
                               Jacobi sweeps on order-64 blocks; 0 redoes every block; must be >= 0 */
} scs_settings;

typedef struct {
    int32_t status;      /* SCS_SOLVED ... SCS_NUMERICAL */
    int32_t iters;       /* outer iterations (all phases) */
    int32_t k0, k1, k2, backtracks;
    int64_t cg_iters;
    double pr, dr, gap, ic, uc; /* Sec. 4.3, evaluated in FP64 on the final iterate */
    double pobj, dobj;   /* <c,x> and -<b,y> */
    double setup_s, solve_s;
    double err_vs_fp64;  /* unused by the library (0); benchmarks fill it */
    int32_t iters_fp32;  /* outer iterations of the FP32 phase (SCS_MIXED) */
    int32_t device_error;/* nonzero if a device barrier timed out */
    double kernel_s[2];  /* device time of the solver launch of the FP64 [0] and FP32 [1] phase
                            (CUDA events on the work's stream) */
    int64_t mat_passes[2]; /* passes over A or A^T (one SpMV each) in the FP64 [0] / FP32 [1] phase */
    int64_t cg_iters_fp32; /* CG iterations of the FP32 phase */
    double psd_resid_fp32; /* largest FP64-evaluated ||X V - V L||_F / ||X||_F of the FP32 PSD
                              eigensolves (SCS_MIXED with PSD cones) */
    int32_t threads_per_block; /* launch shape used (batches: chosen by the autotuner unless set) */
    int32_t warm_fallback_taken; /* 1 if the warm start was abandoned for the cold start */
    double kkt_fp32;        /* max(pr, dr, gap) of the FP32 phase's last termination test, evaluated
                               on FP32 data (SCS_MIXED; 0 otherwise) */
    int64_t mat_passes_ir;  /* FP32 passes over A or A^T of the FP64 phase's refinement corrections */
    int64_t cg_iters_ir;    /* FP32 CG iterations of those corrections (also counted in cg_iters) */
    int64_t ir_sweeps;      /* correction solves of the FP64 phase's iterative refinement */
    double batch_device_s;  /* scs_batch_solve: device time of the whole batch solve (both phases,
                               hand-over, packing, copies to the host staging), CUDA events on the
                               stream it runs on; the same in every instance's info */
    int32_t team;           /* execution team that ran: SCS_TEAM_BLOCK (k_block) or SCS_TEAM_GRID (k_grid) */
    double part_s[2][5];    /* device time of the parts of Algorithm 1 in the FP64 [0] and FP32 [1]
                               phase: termination tests, directions, linear solves (all), the CG
                               loops inside them, the rest (steps, line searches, projections) */
    int64_t psd_redo_fp32;  /* PSD projections of the FP32 phase recomputed in FP64 (eigen-residual
                               above psd_recheck_tol) */
} scs_info;

typedef struct scs_work scs_work;   /* opaque; owns all device memory of one problem */
typedef struct scs_batch scs_batch; /* opaque; owns all device memory of a batch */

/* Fills *out with the defaults: AA, mem 10, eps 1e-5, c0 0.99, c1 0.99,
 * q 0.99, sigma 1e-2, lambda 1, thetabar 0.1, max_iters 10000, ls_max 20,
 * cg_max 1000, check_every 1, cg_rtol 1e-10, FP64, cold start, auto team. */
int scs_default_settings(scs_settings *out);

/* Validates the data, copies A, b, c to the device, builds the transposed
 * copy of A (CSR of A^T) and precomputes g = M^{-1}(c, b) (one CG solve; the
 * block elimination of (I+Q)^{-1}, Sec. 4.1).  cuda_stream may be NULL (the
 * legacy default stream).  On success *out owns the device memory. */
int scs_setup(const scs_data *data, const scs_cone *cone, const scs_settings *settings,
              void *cuda_stream, scs_work **out);

/* Runs Algorithm 1 to the settings' tolerance.  x (n), y (m), s (m) receive
 * the solution (Sec. 3.1 recovery: (chi, psi, sigma)/tau); for INFEASIBLE,
 * y holds the certificate scaled to <b,y> = -1 and x, s are NaN; for
 * UNBOUNDED, x and s hold the certificate scaled to <c,x> = -1 and y is NaN.
 * Any of x, y, s, info may be NULL.  Synchronises the work's stream. */
int scs_solve(scs_work *work, double *x, double *y, double *s, scs_info *info);

/* Replaces b (m) and/or c (n) of a set-up problem (NULL keeps the old one)
 * and recomputes g; A and the cones stay.  For parametric families. */
int scs_update_bc(scs_work *work, const double *b, const double *c);

/* The final HSDE iterate u (N values) of the last scs_solve, for warm starts
 * and checkpoint/resume (any u0 converges, Sec. 4.5). */
int scs_get_u(scs_work *work, double *u);

/* u0 of the next solves: u (N values, host or device) is copied now; NULL
 * returns to the cold start (0, 0, 1).  Combined with settings->warm_fallback. */
int scs_set_warm(scs_work *work, const double *u);

/* Relative primal residual, dual residual and duality gap of Sec. 4.3 for a
 * caller's candidate (x, y, s) on the work's data:
 *   out[0] = ||A x + s - b|| / (1 + ||b||),  out[1] = ||A^T y + c|| / (1 + ||c||),
 *   out[2] = |<c,x> + <b,y>| / (1 + |<c,x>| + |<b,y>|).
 * x (n), y (m), s (m) and out (3) may be host or device pointers.  Cone
 * membership of s and y is not checked.  Synchronises the work's stream. */
int scs_residuals(scs_work *work, const double *x, const double *y, const double *s, double *out);

/* The same three numbers as scs_residuals (up to rounding: the sums of A^T y
 * are accumulated with atomic additions, whose order varies from call to
 * call), for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a service of the library.  It needs no scs_work (whose
 * setup allocates) and never calls cudaMalloc or cudaFree: its only scratch
 * -- the vector A^T y and per-block partial sums -- is a static device array
 * of 8 MiB + 56 KiB that every GPU loading this library holds until the
 * process exits.  Typical callers: real-time or embedded loops that forbid
 * allocation after start-up, since cudaMalloc may block and synchronise the
 * device; hosts whose device memory belongs to another allocator or memory
 * pool, which a second allocator would fragment or exhaust.
 *
 * Every pointer is a device pointer: A as CSR (Ap[m+1] int64, Ai[nnz] int32
 * column indices in [0,n), Ax[nnz]), b (m), c (n), x (n), y (m), s (m), and
 * out (3 doubles: pr, dr, gap).  n above 1048576 is rejected with SCS_EINVAL
 * (message in scs_last_error(NULL)).  A column index outside [0,n) is skipped
 * by the kernel and makes all three outputs NaN; the row pointers must be
 * nondecreasing and within Ai and Ax (not checked).  The work is queued on
 * cuda_stream (NULL: legacy default stream) and the call returns without
 * synchronising.  The scratch array's device address is looked up once per
 * CUDA context: the first call on each device does it, with that device
 * current (and again after cudaDeviceReset, which creates a new context);
 * make that first call before any stream capture.  All calls share the one
 * scratch array and it keeps the last call's contents (its A^T y part is
 * cleared at the start of each call), so calls whose work may overlap on the
 * GPU -- from different streams or threads -- race and must be serialised. */
int scs_residuals_noalloc(int32_t m, int32_t n, const int64_t *Ap, const int32_t *Ai, const double *Ax,
                          const double *b, const double *c, const double *x, const double *y,
                          const double *s, double *out, void *cuda_stream);

/* --- single operators of Eq. (drs), for checking one step at a time ------ */
/* out = (I+Q)^{-1} r on N-vectors (Sec. 4.1, linear-system step of Eq. drs).
 * Uses and updates the work's CG warm start of slot 0 (u~) or 1 (d~).  slot
 * + 2 (works set up with SCS_MIXED): the FP64 solve by iterative refinement
 * as the FP64 phase runs it (FP64 residuals, FP32 CG corrections). */
int scs_linsys(scs_work *work, const double *r, double *out, int32_t slot);
/* out = Pi_C(v), C = R^n x K* x R_+ (Sec. 3.1; projection step of Eq. drs). */
int scs_project_cone(scs_work *work, const double *v, double *out);
/* The same projection in the bulk precision SCS_FP64 or (works set up with
 * SCS_MIXED) as the FP32 phase runs it -- FP32 data, FP32 Jacobi eigensolves
 * with the FP64 recheck and redo of psd_recheck_tol.  stats (may be NULL)
 * receives [0] the largest relative eigen-residual of the FP32 eigensolves
 * and [1] the number of PSD blocks decomposed again in FP64 (both 0 for
 * SCS_FP64).  Pointers host or device; SCS_EINVAL on bad arguments. */
int scs_project_cone_prec(scs_work *work, int32_t precision, const double *v, double *out, double *stats);
/* Tu = u + Pi_C(2u~ - u) - u~ and Ru = u - Tu (Sec. 4.1-4.2); either may be NULL. */
int scs_apply_T(scs_work *work, const double *u, double *Tu, double *Ru);

/* Sparse products of the solver's own matrix copies, in the bulk precision
 * SCS_FP64 or (works set up with SCS_MIXED) the FP32 copy, for checking the
 * products on their own -- every CG iteration of Sec. 4.1 is one A and one
 * A^T product.  op 0: out (m) = A in (n); op 1: out (n) = A^T in (m); op 2:
 * out = A^T in and out2 = A^T in2 (in, in2 of m entries) in one fused pass.
 * Results are widened to FP64; pointers host or device.  Overwrites the
 * work's scratch vectors; SCS_EINVAL on bad arguments. */
int scs_spmv(scs_work *work, int32_t precision, int32_t op, const double *in, const double *in2, double *out,
             double *out2);

/* Host-only diagnostic of the column-blocked layout the grid team uses for
 * large matrices (no counterpart in the paper; no GPU needed): builds the
 * layout of the rows x cols CSR matrix (Ap, Ai, Ax) for `ctas` CTAs of
 * `compute_warps` compute warps, elem_bytes 4 (FP32 copy) or 8 (FP64),
 * `vectors` 1 or 2 multiplied vectors, smem_bytes of dynamic shared memory,
 * checks its invariants, and replays y = A x (x: cols, y: rows, host) the way
 * the device loop walks the layout, in FP64.  stats[8] (host): [0] violated
 * invariants, [1] column blocks (0: the layout does not fit), [2] block
 * width, [3] lanes per row, [4] stored entries, [5] dynamic shared memory,
 * [6] ring stages, [7] metadata words per segment.  SCS_EINVAL on bad input. */
int scs_cb_layout_check(int32_t rows, int32_t cols, const int64_t *Ap, const int32_t *Ai, const double *Ax,
                        int32_t ctas, int32_t compute_warps, int32_t elem_bytes, int32_t vectors,
                        int64_t smem_bytes, const double *x, double *y, int64_t *stats);
/* The same for the two-dimensional tiled layout (tiles of a row block times
 * a column block, one per CTA, the column block's slice of x resident in
 * shared memory, partial sums per column block added in block order by a
 * second pass): builds it (forced, whatever the size), checks its invariants
 * and replays y = A x as the tile passes and the second pass compute it, in
 * FP64.  stats[8]: [0] violated invariants, [1] column blocks (0: no split
 * fits), [2] row blocks, [3] lanes per row, [4] stored entries, [5] dynamic
 * shared memory, [6] chunks, [7] metadata words per chunk.  SCS_EINVAL on
 * bad input. */
int scs_tile_layout_check(int32_t rows, int32_t cols, const int64_t *Ap, const int32_t *Ai, const double *Ax,
                          int32_t ctas, int32_t compute_warps, int32_t elem_bytes, int32_t vectors,
                          int64_t smem_bytes, const double *x, double *y, int64_t *stats);

/* Device-side timing (globaltimer between team barriers, inside one launch)
 * of the solver's building blocks on this problem, for roofline measurement:
 * ns[0] one product with A, ns[1] one with A^T, ns[2] one team barrier,
 * ns[3] one team reduction, ns[4] one CG iteration; each averaged over reps.
 * precision SCS_FP64 times the FP64 data; SCS_MIXED the FP32 copy (only on
 * works set up with SCS_MIXED).  Overwrites the work's scratch vectors. */
int scs_profile(scs_work *work, int32_t precision, int32_t reps, double *ns);

/* Frees everything owned by work; NULL-safe. */
void scs_finish(scs_work *work);

/* Message of the last error on work, or of the calling thread when work is NULL. */
const char *scs_last_error(const scs_work *work);

/* --- batched solves ------------------------------------------------------ */
/* B independent instances of any sizes, solved by one persistent launch (per
 * precision phase) in which each thread block takes instances from a queue,
 * largest first.  The settings apply to every instance (team is ignored: one
 * block each).  With settings->threads = 0 and B >= 64 the setup times the
 * first solve phase on a sample of instances for 128, 256, 512 and 1024 threads
 * per block and keeps the fastest; the sample holds enough instances for two
 * waves of the largest resident grid among the four (at most all B). */
int scs_batch_setup(int32_t B, const scs_data *const *data, const scs_cone *const *cones,
                    const scs_settings *settings, void *cuda_stream, scs_batch **out);
/* x[i], y[i], s[i] (host pointers; any may be NULL, as may the arrays)
 * receive instance i's result as in scs_solve; infos may be NULL or hold B
 * entries.  Results are gathered on the device and copied back in one
 * transfer.  The device work of a solve (both precision phases, the hand-
 * over, the packing and the copies) is captured once into a CUDA graph on a
 * stream the batch owns and replayed by one graph launch per solve, ordered
 * after the work already queued on cuda_stream (captured again when the
 * warm-start mode changes); if capture is unavailable it is enqueued on
 * cuda_stream directly. */
int scs_batch_solve(scs_batch *batch, double *const *x, double *const *y, double *const *s,
                    scs_info *infos);
void scs_batch_finish(scs_batch *batch);
/* A batch of B instances sharing the matrix A and cones of *data (its b and
 * c are ignored) with instance i's b[i] (m) and c[i] (n): the matrix is
 * prepared and stored once; everything else is as scs_batch_setup.  For
 * parametric families such as the LASSO family of a fixed design matrix. */
int scs_batch_setup_shared(int32_t B, const scs_data *data, const scs_cone *cone, const double *const *b,
                           const double *const *c, const scs_settings *settings, void *cuda_stream,
                           scs_batch **out);
/* Warm starts for the next solves of the batch: u[i] (N_i values, host or
 * device) is instance i's u0; u = NULL returns to cold starts.  Combined
 * with settings->warm_fallback. */
int scs_batch_set_warm(scs_batch *batch, const double *const *u);
/* One-shot: setup, solve, finish. */
int scs_solve_batch(int32_t B, const scs_data *const *data, const scs_cone *const *cones,
                    const scs_settings *settings, void *cuda_stream, double *const *x,
                    double *const *y, double *const *s, scs_info *infos);

#ifdef __cplusplus
}
#endif
#endif /* SUPERSCS_H */
