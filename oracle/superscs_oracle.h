/*
 * superscs_oracle.h -- plain, slow, FP64 CPU reference of SuperSCS.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file; only the test-suite, the package's smoke check and the
 * CPU-baseline leg of the benchmark use it.  It shares no code, header,
 * table or constant with the CUDA implementation.
 *
 * Notation follows Sopasakis, Menounou, Patrinos, "SuperSCS: fast and accurate
 * large-scale conic optimization" (arXiv 1903.06477):
 *   primal   (P)   min <c,x>  s.t.  b - A x = s,  s in K                 (Sec. 3)
 *   dual     (D)   min <b,y>  s.t.  y in K*,  A^T y + c = 0              (Sec. 3)
 *   HSDE     u = (chi, psi, tau),  Q = [0 A^T c; -A 0 b; -c^T -b^T 0]   (Sec. 3.1)
 *   DRS      u~ = (I+Q)^{-1} u,  u_ = Pi_C(2u~ - u),  u+ = u + u_ - u~   (Eq. drs)
 *   T, R     Tu = u + Pi_C(2u~-u) - u~,  R = I - T                      (Sec. 4.1-4.2)
 *   SuperMann with K0/K1/K2 steps                                        (Algorithm 1)
 *   restarted Broyden directions                                         (Algorithm 2)
 *   Anderson's acceleration                                              (Sec. 4.4.2)
 *   termination and certificates                                         (Sec. 4.3)
 *
 * Cone rows of s are ordered [ f zero | l orthant | q SOCs... | s PSDs... |
 * ep primal exponential cones | ed dual exponential cones ] (3 rows each).
 * A is CSR with m rows: Ap[m+1] (int64), Ai[nnz] (int32), Ax[nnz].
 *
 * Parity status of each function is stated in the tests that pin it.  The
 * iterate path of Algorithm 1 is pinned step by step where every step takes
 * the same branch: all K0 (Anderson acceleration in Walker and Ni's form, or
 * a dense safeguarded Broyden iteration) and all K2 (the KM iteration).  Paths
 * that mix K1, K2 and backtracking are "parity unpinned": only their end
 * results and branch invariants are pinned.
 */
#ifndef SUPERSCS_ORACLE_H
#define SUPERSCS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n, m;
    const int64_t *Ap;
    const int32_t *Ai;
    const double *Ax;
    const double *b, *c;
    int32_t f, l;
    int32_t nq;
    const int32_t *q;
    int32_t ns;
    const int32_t *s;
    int32_t ep, ed;  /* primal / dual exponential cones, 3 rows each, after the PSD rows */
} orc_problem;

/* ORC_DIR_AA_QR: Anderson's acceleration with its least-squares problem solved
 * through a QR factorisation of the window of residual differences, updated
 * as pairs enter (Gram-Schmidt) and leave (Givens rotations) -- Sec. 4.4. */
enum { ORC_DIR_AA = 0, ORC_DIR_RB = 1, ORC_DIR_NONE = 2, ORC_DIR_AA_QR = 3 };

typedef struct {
    int32_t direction;   /* ORC_DIR_AA | ORC_DIR_RB | ORC_DIR_NONE (d = 0: pure KM) */
    int32_t mem;
    double eps, c0, c1, q, sigma, lambda, thetabar;
    int32_t max_iters, ls_max, cg_max, check_every;
    double cg_rtol;
    double aa_reg;
    const double *warm_u; /* N = n+m+1 values or NULL for u0 = (0,0,1) */
    double cg_adapt;      /* > 0: inside the loop CG also stops at ||res|| <= cg_adapt ||Ru|| */
} orc_settings;

enum {
    ORC_SOLVED = 1,
    ORC_INFEASIBLE = -1,
    ORC_UNBOUNDED = -2,
    ORC_MAX_ITERS = -3,
    ORC_NUMERICAL = -5
};

typedef struct {
    int32_t status, iters, k0, k1, k2, backtracks;
    int64_t cg_iters;
    double pr, dr, gap, ic, uc, pobj, dobj, nRu;
} orc_info;

/* Optional per-iteration trace of Algorithm 1 (arrays of length cap). */
typedef struct {
    int32_t cap;
    int32_t len;
    double *nRu;       /* ||R u^nu|| at the start of iteration nu            */
    int32_t *step;     /* 0 = K0, 1 = K1, 2 = K2                             */
    double *alpha;     /* accepted alpha (K1/K2), 1 for K0                   */
    double *u_dist;    /* ||u^{nu+1} - ustar||, only if ustar != NULL        */
    const double *ustar;
} orc_trace;

typedef struct orc_work orc_work;

/* --- cones (Sec. 2) ------------------------------------------------------ */
/* Exponential cone, cone (v) of Sec. 2, in the paper's element order:
 * K^e = cl{(x1, x2, x3) : x1 >= x2 exp(x3 / x2), x2 > 0}.  orc_proj_exp
 * projects v (3 values, in place) on K^e, orc_proj_exp_dual on its dual cone
 * (K^e)* = cl{(y1, y2, y3) : y3 < 0, -y3 exp(y2 / y3) <= e y1}; the
 * membership tests return 1 inside (closure), 0 outside. */
void orc_proj_exp(double *v);
void orc_proj_exp_dual(double *v);
int  orc_in_exp(const double *v, double tol);
int  orc_in_exp_dual(const double *v, double tol);
void orc_proj_soc(double *z, int32_t dim);
int  orc_jacobi_eig(int32_t d, const double *Xin, double *lam, double *V);
int  orc_proj_psd(double *v, int32_t d);
void orc_svec_to_mat(int32_t d, const double *v, double *X);
void orc_mat_to_svec(int32_t d, const double *X, double *v);
int  orc_proj_dual_cone(const orc_problem *P, double *v);
int  orc_proj_primal_cone(const orc_problem *P, double *v);
int  orc_proj_C(const orc_problem *P, const double *v, double *out);

/* --- work object: holds g = M^{-1} h and CG warm starts --------------------- */
orc_work *orc_setup(const orc_problem *P, const orc_settings *S);
void orc_finish(orc_work *W);
/* out = (I+Q)^{-1} r, both of length N; slot 0 = u~ warm start, slot 1 = d~ */
int  orc_linsys(orc_work *W, const double *r, double *out, int32_t slot, int32_t *cg_iters);
/* Tu and Ru for one u (either output may be NULL); uses the u~ slot */
int  orc_apply_T(orc_work *W, const double *u, double *Tu, double *Ru);
/* Sec. 4.3 on a triple (u, u~, u_); fills info pr/dr/gap/ic/uc and returns status (0 = continue) */
int  orc_termination(orc_work *W, const double *u, const double *ut, const double *ub,
                     double eps, orc_info *info);
/* Algorithm 1; x[n], y[m], s[m], u_out[N] (u_out may be NULL, trace may be NULL) */
int  orc_solve(orc_work *W, double *x, double *y, double *s, double *u_out,
               orc_info *info, orc_trace *trace);

/* --- directions, stateful, for pins (Sec. 4.4) ---------------------------- */
typedef struct orc_dir orc_dir;
orc_dir *orc_dir_new(int32_t kind, int64_t N, int32_t mem, double thetabar, double aa_reg);
void orc_dir_free(orc_dir *D);
/* have_pair = 0: d = -Ru; else uses pair (z, xi) = (w-u, Rw-Ru) of the previous iteration */
int  orc_dir_compute(orc_dir *D, const double *Ru, const double *z, const double *xi,
                     int32_t have_pair, double *d);
int32_t orc_dir_count(const orc_dir *D);

#ifdef __cplusplus
}
#endif
#endif
