/*
 * superscs_oracle.c -- plain, slow, FP64 CPU reference of SuperSCS
 * (Sopasakis, Menounou, Patrinos, arXiv 1903.06477).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg.  Never called by the product path, and it
 * shares nothing with the CUDA implementation.
 *
 * Every routine is written as the paper states it, with plain loops and no
 * blocking or fusion.  Where the paper is silent, the reading taken is given
 * in the comment above the routine.
 */
#define _GNU_SOURCE
#include "superscs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define SQRT2 1.41421356237309504880

/* ------------------------------------------------------------------------ */
/* plain vector helpers                                                     */
/* ------------------------------------------------------------------------ */
static double vdot(const double *a, const double *b, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}
static double vnorm(const double *a, int64_t n) { return sqrt(vdot(a, a, n)); }

/* y = A x  (A: m x n CSR) */
static void A_mul(const orc_problem *P, const double *x, double *y)
{
    for (int32_t i = 0; i < P->m; ++i) {
        double s = 0.0;
        for (int64_t k = P->Ap[i]; k < P->Ap[i + 1]; ++k) s += P->Ax[k] * x[P->Ai[k]];
        y[i] = s;
    }
}
/* x = A^T y, by scattering each CSR row (no transposed copy: this is the definition) */
static void AT_mul(const orc_problem *P, const double *y, double *x)
{
    for (int32_t j = 0; j < P->n; ++j) x[j] = 0.0;
    for (int32_t i = 0; i < P->m; ++i)
        for (int64_t k = P->Ap[i]; k < P->Ap[i + 1]; ++k) x[P->Ai[k]] += P->Ax[k] * y[i];
}

/* ------------------------------------------------------------------------ */
/* cones (Sec. 2)                                                            */
/* ------------------------------------------------------------------------ */

/* Second-order cone K^q = {(x,t) : ||x||_2 <= t}, t stored LAST.  Closed-form
 * Euclidean projection: identity inside, 0 in the polar cone, otherwise
 * ((||x||+t)/(2||x||)) (x, ||x||). */
void orc_proj_soc(double *z, int32_t dim)
{
    if (dim <= 0) return;
    double t = z[dim - 1];
    double nx = vnorm(z, dim - 1);
    if (nx <= t) return;
    if (nx <= -t) {
        for (int32_t i = 0; i < dim; ++i) z[i] = 0.0;
        return;
    }
    double a = (nx + t) / (2.0 * nx);
    for (int32_t i = 0; i < dim - 1; ++i) z[i] *= a;
    z[dim - 1] = a * nx;
}

/* Exponential cone K^e = cl{(x1,x2,x3) : x1 >= x2 exp(x3/x2), x2 > 0} (Sec. 2,
 * cone (v)).  Below a point is named by (r, s, t) = (x3, x2, x1), so K^e =
 * cl{s exp(r/s) <= t, s > 0} and its dual (K^e)* = cl{(u, v, w) : u < 0,
 * -u exp(v/u) <= e w} in the same roles (u = y3, v = y2, w = y1).
 *
 * Projection of a point outside K^e and outside its polar -(K^e)*: the
 * nearest point of K^e lies on its boundary, which is the face {s = 0, r <= 0,
 * t >= 0} together with the rays {c (rho, 1, e^rho) : c >= 0}.  The nearest
 * point of the face is (min(r,0), 0, max(t,0)).  On the ray of slope rho the
 * nearest point is c a with a = (rho, 1, e^rho) and c = <v,a>/|a|^2; the
 * distance is stationary in rho exactly where
 *   F(rho) = r (1 + (1-rho) e^{2 rho}) - s (rho + e^{2 rho}) + t e^rho (rho^2 - rho + 1)
 * vanishes (the derivative of <v,a>^2/|a|^2, cleared of positive factors).
 * The oracle collects every candidate -- the face point, the origin, and the
 * point of every root of F with c > 0, found by scanning rho on a fine grid
 * and bisecting each sign change -- all of which lie in K^e, and returns the
 * nearest.  F is evaluated as F e^{-2 rho} for rho > 0 (same sign, no
 * overflow); roots beyond the grid are bracketed by doubling. */
static double exp_F(double rho, double r, double s, double t)
{
    if (rho <= 0.0) {
        const double e = exp(rho), e2 = e * e;
        return r * (1.0 + (1.0 - rho) * e2) - s * (rho + e2) + t * e * (rho * rho - rho + 1.0);
    }
    const double em = exp(-rho), em2 = em * em;
    return r * ((1.0 - rho) + em2) - s * (rho * em2 + 1.0) + t * em * (rho * rho - rho + 1.0);
}

/* the point c a of the ray of slope rho nearest to (r,s,t), as (r,s,t); 0 if c <= 0 */
static int exp_ray_point(double rho, double r, double s, double t, double *pr, double *ps, double *pt)
{
    double a0, a1, a2;  /* a scaled by max(1, e^rho)^-1 */
    if (rho <= 0.0) { a0 = rho; a1 = 1.0; a2 = exp(rho); }
    else { const double em = exp(-rho); a0 = rho * em; a1 = em; a2 = 1.0; }
    const double c = (r * a0 + s * a1 + t * a2) / (a0 * a0 + a1 * a1 + a2 * a2);
    if (!(c > 0.0)) return 0;
    *pr = c * a0; *ps = c * a1; *pt = c * a2;
    return 1;
}

static double exp_bisect(double lo, double hi, double r, double s, double t)
{
    double flo = exp_F(lo, r, s, t);
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double fm = exp_F(mid, r, s, t);
        if (fm == 0.0) return mid;
        if ((fm > 0.0) == (flo > 0.0)) { lo = mid; flo = fm; } else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static int exp_member(double r, double s, double t, double tol)
{
    if (s > 0.0) return s * exp(r / s) <= t + tol;   /* exp overflow gives +inf: outside */
    return s >= -tol && r <= tol && t >= -tol;
}
static int exp_dual_member(double u, double v, double w, double tol)
{
    if (u < 0.0) return -u * exp(v / u) <= M_E * w + tol;
    return u <= tol && v >= -tol && w >= -tol;
}
int orc_in_exp(const double *x, double tol) { return exp_member(x[2], x[1], x[0], tol); }
int orc_in_exp_dual(const double *y, double tol) { return exp_dual_member(y[2], y[1], y[0], tol); }

void orc_proj_exp(double *x)
{
    const double r = x[2], s = x[1], t = x[0];
    if (exp_member(r, s, t, 0.0)) return;
    if (exp_dual_member(-r, -s, -t, 0.0)) { x[0] = x[1] = x[2] = 0.0; return; }  /* v in the polar cone */
    if (r <= 0.0 && s <= 0.0) { x[0] = t > 0.0 ? t : 0.0; x[1] = 0.0; return; }
    /* candidates: the origin, the face point, the ray points at the roots of F */
    double best_r = 0.0, best_s = 0.0, best_t = 0.0;
    double best_d = r * r + s * s + t * t;
    {
        const double fr = r < 0.0 ? r : 0.0, ft = t > 0.0 ? t : 0.0;
        const double d = (r - fr) * (r - fr) + s * s + (t - ft) * (t - ft);
        if (d < best_d) { best_d = d; best_r = fr; best_s = 0.0; best_t = ft; }
    }
    const double L = 60.0, h = 0.05;
    const int npts = (int)(2.0 * L / h + 0.5) + 1;
    double roots[64];
    int nr = 0;
    double prev_x = -L, prev_f = exp_F(-L, r, s, t);
    /* below the grid: F ~ r - s rho, one sign change at most */
    {
        double lo = -L;
        for (int k = 0; k < 1100 && nr < 64; ++k) {
            const double lo2 = 2.0 * lo;
            if ((exp_F(lo2, r, s, t) > 0.0) != (exp_F(lo, r, s, t) > 0.0)) {
                roots[nr++] = exp_bisect(lo2, lo, r, s, t);
                break;
            }
            lo = lo2;
            if (!isfinite(lo)) break;
        }
    }
    for (int k = 1; k < npts && nr < 64; ++k) {
        const double xk = -L + h * k;
        const double fk = exp_F(xk, r, s, t);
        if (fk == 0.0) roots[nr++] = xk;
        else if ((fk > 0.0) != (prev_f > 0.0) && prev_f != 0.0) roots[nr++] = exp_bisect(prev_x, xk, r, s, t);
        prev_x = xk;
        prev_f = fk;
    }
    /* above the grid: F e^{-2 rho} ~ r (1 - rho) - s, one sign change at most */
    {
        double hi = L;
        for (int k = 0; k < 1100 && nr < 64; ++k) {
            const double hi2 = 2.0 * hi;
            if ((exp_F(hi2, r, s, t) > 0.0) != (exp_F(hi, r, s, t) > 0.0)) {
                roots[nr++] = exp_bisect(hi, hi2, r, s, t);
                break;
            }
            hi = hi2;
            if (!isfinite(hi)) break;
        }
    }
    for (int k = 0; k < nr; ++k) {
        double pr, ps, pt;
        if (!exp_ray_point(roots[k], r, s, t, &pr, &ps, &pt)) continue;
        const double d = (r - pr) * (r - pr) + (s - ps) * (s - ps) + (t - pt) * (t - pt);
        if (d < best_d) { best_d = d; best_r = pr; best_s = ps; best_t = pt; }
    }
    x[0] = best_t;
    x[1] = best_s;
    x[2] = best_r;
}

/* Moreau: Pi_{K*}(v) = v + Pi_K(-v), since the polar of K* is -K */
void orc_proj_exp_dual(double *v)
{
    double w[3] = {-v[0], -v[1], -v[2]};
    orc_proj_exp(w);
    v[0] += w[0];
    v[1] += w[1];
    v[2] += w[2];
}

/* svec index of entry (i, j), i >= j: lower triangle stored column by column
 * (the mat map of Sec. 2: x_1..x_n is column 1, x_{n+1}..x_{2n-1} column 2, ...) */
static int64_t svec_idx(int32_t d, int32_t i, int32_t j)
{
    return (int64_t)j * d - (int64_t)j * (j - 1) / 2 + (i - j);
}

/* mat(v): diagonal entries as stored, off-diagonal entries divided by sqrt(2) */
void orc_svec_to_mat(int32_t d, const double *v, double *X)
{
    for (int32_t j = 0; j < d; ++j)
        for (int32_t i = j; i < d; ++i) {
            double e = v[svec_idx(d, i, j)];
            if (i != j) e /= SQRT2;
            X[(int64_t)i * d + j] = e;
            X[(int64_t)j * d + i] = e;
        }
}

/* inverse of mat: off-diagonal entries multiplied by sqrt(2) */
void orc_mat_to_svec(int32_t d, const double *X, double *v)
{
    for (int32_t j = 0; j < d; ++j)
        for (int32_t i = j; i < d; ++i) {
            double e = 0.5 * (X[(int64_t)i * d + j] + X[(int64_t)j * d + i]);
            v[svec_idx(d, i, j)] = (i == j) ? e : SQRT2 * e;
        }
}

/* Textbook cyclic Jacobi eigenvalue method for a symmetric d x d matrix
 * (row-major).  Returns eigenvalues lam[d] and eigenvectors as the columns of
 * V (row-major, V[i*d+k] = component i of vector k).  Sweeps all (p,q) pairs
 * in row order until the off-diagonal Frobenius mass is below 1e-30 of the
 * total, at most 100 sweeps. */
int orc_jacobi_eig(int32_t d, const double *Xin, double *lam, double *V)
{
    double *X = (double *)malloc(sizeof(double) * (size_t)d * d);
    if (!X) return -1;
    memcpy(X, Xin, sizeof(double) * (size_t)d * d);
    for (int32_t i = 0; i < d; ++i)
        for (int32_t k = 0; k < d; ++k) V[(int64_t)i * d + k] = (i == k) ? 1.0 : 0.0;

    double total = 0.0;
    for (int64_t i = 0; i < (int64_t)d * d; ++i) total += X[i] * X[i];

    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int32_t p = 0; p < d; ++p)
            for (int32_t q = p + 1; q < d; ++q) off += 2.0 * X[(int64_t)p * d + q] * X[(int64_t)p * d + q];
        if (off <= 1e-30 * total || off == 0.0) break;
        for (int32_t p = 0; p < d - 1; ++p) {
            for (int32_t q = p + 1; q < d; ++q) {
                double apq = X[(int64_t)p * d + q];
                if (apq == 0.0) continue;
                double app = X[(int64_t)p * d + p], aqq = X[(int64_t)q * d + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t;
                if (fabs(theta) > 1e150)
                    t = 0.5 / theta;
                else
                    t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* X <- J^T X J with J the rotation in the (p,q) plane */
                for (int32_t k = 0; k < d; ++k) {
                    double xkp = X[(int64_t)k * d + p], xkq = X[(int64_t)k * d + q];
                    X[(int64_t)k * d + p] = c * xkp - s * xkq;
                    X[(int64_t)k * d + q] = s * xkp + c * xkq;
                }
                for (int32_t k = 0; k < d; ++k) {
                    double xpk = X[(int64_t)p * d + k], xqk = X[(int64_t)q * d + k];
                    X[(int64_t)p * d + k] = c * xpk - s * xqk;
                    X[(int64_t)q * d + k] = s * xpk + c * xqk;
                }
                for (int32_t k = 0; k < d; ++k) {
                    double vkp = V[(int64_t)k * d + p], vkq = V[(int64_t)k * d + q];
                    V[(int64_t)k * d + p] = c * vkp - s * vkq;
                    V[(int64_t)k * d + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int32_t i = 0; i < d; ++i) lam[i] = X[(int64_t)i * d + i];
    free(X);
    return 0;
}

/* PSD cone K^s on svec vectors: Pi(v) = svec(V max(Lambda,0) V^T) with
 * mat(v) = V Lambda V^T. */
int orc_proj_psd(double *v, int32_t d)
{
    if (d <= 0) return 0;
    size_t dd = (size_t)d * d;
    double *X = (double *)malloc(sizeof(double) * dd);
    double *V = (double *)malloc(sizeof(double) * dd);
    double *lam = (double *)malloc(sizeof(double) * (size_t)d);
    if (!X || !V || !lam) { free(X); free(V); free(lam); return -1; }
    orc_svec_to_mat(d, v, X);
    if (orc_jacobi_eig(d, X, lam, V) != 0) { free(X); free(V); free(lam); return -1; }
    for (int32_t i = 0; i < d; ++i)
        for (int32_t j = 0; j < d; ++j) {
            double s = 0.0;
            for (int32_t k = 0; k < d; ++k)
                if (lam[k] > 0.0) s += V[(int64_t)i * d + k] * lam[k] * V[(int64_t)j * d + k];
            X[(int64_t)i * d + j] = s;
        }
    orc_mat_to_svec(d, X, v);
    free(X); free(V); free(lam);
    return 0;
}

static int64_t cone_rows(const orc_problem *P)
{
    int64_t r = (int64_t)P->f + P->l;
    for (int32_t i = 0; i < P->nq; ++i) r += P->q[i];
    for (int32_t i = 0; i < P->ns; ++i) r += (int64_t)P->s[i] * (P->s[i] + 1) / 2;
    r += 3 * (int64_t)P->ep + 3 * (int64_t)P->ed;
    return r;
}

/* Projection on K (primal = 0) or K* (dual = 1) over rows [f | l | q | s | ep | ed].
 * The zero cone's dual is the free cone, so its rows are set to 0 for K and
 * left untouched for K*; orthant, SOC and PSD cones are self-dual. */
static int proj_cone(const orc_problem *P, double *v, int dual)
{
    int64_t o = 0;
    for (int32_t i = 0; i < P->f; ++i, ++o)
        if (!dual) v[o] = 0.0;
    for (int32_t i = 0; i < P->l; ++i, ++o)
        if (v[o] < 0.0) v[o] = 0.0;
    for (int32_t k = 0; k < P->nq; ++k) {
        orc_proj_soc(v + o, P->q[k]);
        o += P->q[k];
    }
    for (int32_t k = 0; k < P->ns; ++k) {
        if (orc_proj_psd(v + o, P->s[k]) != 0) return -1;
        o += (int64_t)P->s[k] * (P->s[k] + 1) / 2;
    }
    /* the exponential cone is not self-dual: a primal block of K projects on
     * K^e and, in K*, on (K^e)*; a dual block the other way round */
    for (int32_t k = 0; k < P->ep; ++k, o += 3) {
        if (dual) orc_proj_exp_dual(v + o); else orc_proj_exp(v + o);
    }
    for (int32_t k = 0; k < P->ed; ++k, o += 3) {
        if (dual) orc_proj_exp(v + o); else orc_proj_exp_dual(v + o);
    }
    return 0;
}
int orc_proj_dual_cone(const orc_problem *P, double *v) { return proj_cone(P, v, 1); }
int orc_proj_primal_cone(const orc_problem *P, double *v) { return proj_cone(P, v, 0); }

/* Pi_C with C = R^n x K* x R_+ (Sec. 3.1) on an N-vector */
int orc_proj_C(const orc_problem *P, const double *v, double *out)
{
    int64_t N = (int64_t)P->n + P->m + 1;
    if (out != v) memcpy(out, v, sizeof(double) * (size_t)N);
    if (proj_cone(P, out + P->n, 1) != 0) return -1;
    if (out[N - 1] < 0.0) out[N - 1] = 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* (I+Q)^{-1} by block elimination and CG (Sec. 4.1, "indirect" solve)      */
/*                                                                          */
/* The paper only says the system is solved directly or by CG.  Reading    */
/* taken: with M = [I A^T; -A I] and h = (c, b), I+Q = [M h; -h^T 1], so    */
/*   tau = (r_tau + h^T M^{-1} r_xy) / (1 + h^T g),  g = M^{-1} h,          */
/*   (x, y) = M^{-1} r_xy - tau g,                                          */
/* and M^{-1}(a, e) is x = (I + A^T A)^{-1}(a - A^T e), y = e + A x.        */
/* CG stops when ||res|| <= cg_rtol ||rhs|| or after cg_max iterations.     */
/* ------------------------------------------------------------------------ */
struct orc_work {
    orc_problem P;
    orc_settings S;
    int64_t N;
    double *g;        /* n+m */
    double hg;        /* h^T g */
    double *ws[2];    /* CG warm starts (n) for the u~ and d~ systems */
    double *tm, *tn, *r, *p, *q, *rhs; /* scratch */
    int64_t cg_total;
    double atol; /* absolute CG tolerance of the next solves (0 = rtol only) */
};

/* CG on (I + A^T A) x = rhs, x holds the warm start on entry */
static int cg_solve(orc_work *W, const double *rhs, double *x, double rtol, int32_t cg_max)
{
    const orc_problem *P = &W->P;
    int32_t n = P->n;
    double *r = W->r, *p = W->p, *q = W->q, *tm = W->tm;
    double bnorm = vnorm(rhs, n);
    if (bnorm == 0.0) {
        for (int32_t j = 0; j < n; ++j) x[j] = 0.0;
        return 0;
    }
    /* r = rhs - (x + A^T A x) */
    A_mul(P, x, tm);
    AT_mul(P, tm, q);
    for (int32_t j = 0; j < n; ++j) { r[j] = rhs[j] - x[j] - q[j]; p[j] = r[j]; }
    double rr = vdot(r, r, n);
    double tol = rtol * bnorm;
    if (W->atol > tol) tol = W->atol;
    int32_t it = 0;
    if (sqrt(rr) <= tol) return 0;
    for (it = 0; it < cg_max; ++it) {
        A_mul(P, p, tm);
        AT_mul(P, tm, q);
        for (int32_t j = 0; j < n; ++j) q[j] += p[j];
        double pq = vdot(p, q, n);
        double alpha = rr / pq;
        for (int32_t j = 0; j < n; ++j) { x[j] += alpha * p[j]; r[j] -= alpha * q[j]; }
        double rr_new = vdot(r, r, n);
        if (sqrt(rr_new) <= tol) { ++it; break; }
        double beta = rr_new / rr;
        for (int32_t j = 0; j < n; ++j) p[j] = r[j] + beta * p[j];
        rr = rr_new;
    }
    return it;
}

/* (x, y) = M^{-1}(a, e) with x warm-started from ws; out has n+m entries */
static int Minv(orc_work *W, const double *a, const double *e, double *out, double *ws, double rtol,
                int32_t cg_max)
{
    const orc_problem *P = &W->P;
    int32_t n = P->n, m = P->m;
    AT_mul(P, e, W->tn);
    for (int32_t j = 0; j < n; ++j) W->rhs[j] = a[j] - W->tn[j];
    int it = cg_solve(W, W->rhs, ws, rtol, cg_max);
    memcpy(out, ws, sizeof(double) * (size_t)n);
    A_mul(P, ws, W->tm);
    for (int32_t i = 0; i < m; ++i) out[n + i] = e[i] + W->tm[i];
    return it;
}

orc_work *orc_setup(const orc_problem *P, const orc_settings *S)
{
    if (!P || !S || P->n <= 0 || P->m <= 0) return NULL;
    if (cone_rows(P) != P->m) return NULL;
    orc_work *W = (orc_work *)calloc(1, sizeof(orc_work));
    if (!W) return NULL;
    W->P = *P;
    W->S = *S;
    int32_t n = P->n, m = P->m;
    W->N = (int64_t)n + m + 1;
    W->g = (double *)calloc((size_t)(n + m), sizeof(double));
    W->ws[0] = (double *)calloc((size_t)n, sizeof(double));
    W->ws[1] = (double *)calloc((size_t)n, sizeof(double));
    W->tm = (double *)calloc((size_t)m, sizeof(double));
    W->tn = (double *)calloc((size_t)n, sizeof(double));
    W->r = (double *)calloc((size_t)n, sizeof(double));
    W->p = (double *)calloc((size_t)n, sizeof(double));
    W->q = (double *)calloc((size_t)n, sizeof(double));
    W->rhs = (double *)calloc((size_t)n, sizeof(double));
    if (!W->g || !W->ws[0] || !W->ws[1] || !W->tm || !W->tn || !W->r || !W->p || !W->q || !W->rhs) {
        orc_finish(W);
        return NULL;
    }
    /* g = M^{-1} h, h = (c, b), from a zero start */
    double *gx = (double *)calloc((size_t)n, sizeof(double));
    if (!gx) { orc_finish(W); return NULL; }
    int it = Minv(W, P->c, P->b, W->g, gx, S->cg_rtol, S->cg_max > 0 ? 10 * S->cg_max : 10000);
    free(gx);
    W->cg_total += it;
    W->hg = vdot(P->c, W->g, n) + vdot(P->b, W->g + n, m);
    return W;
}

void orc_finish(orc_work *W)
{
    if (!W) return;
    free(W->g); free(W->ws[0]); free(W->ws[1]); free(W->tm); free(W->tn);
    free(W->r); free(W->p); free(W->q); free(W->rhs);
    free(W);
}

int orc_linsys(orc_work *W, const double *r, double *out, int32_t slot, int32_t *cg_iters)
{
    const orc_problem *P = &W->P;
    int32_t n = P->n, m = P->m;
    int64_t N = W->N;
    double *pz = (double *)malloc(sizeof(double) * (size_t)(n + m));
    if (!pz) return -1;
    int it = Minv(W, r, r + n, pz, W->ws[slot ? 1 : 0], W->S.cg_rtol, W->S.cg_max);
    W->cg_total += it;
    if (cg_iters) *cg_iters = it;
    double htp = vdot(P->c, pz, n) + vdot(P->b, pz + n, m);
    double tau = (r[N - 1] + htp) / (1.0 + W->hg);
    for (int64_t i = 0; i < n + m; ++i) out[i] = pz[i] - tau * W->g[i];
    out[N - 1] = tau;
    free(pz);
    return 0;
}

/* u_ = Pi_C(2 u~ - u), Ru = u~ - u_ (Eq. drs, R = I - T) */
static int eval_R(orc_work *W, const double *u, const double *ut, double *ub, double *Ru)
{
    int64_t N = W->N;
    for (int64_t i = 0; i < N; ++i) ub[i] = 2.0 * ut[i] - u[i];
    if (orc_proj_C(&W->P, ub, ub) != 0) return -1;
    for (int64_t i = 0; i < N; ++i) Ru[i] = ut[i] - ub[i];
    return 0;
}

int orc_apply_T(orc_work *W, const double *u, double *Tu, double *Ru)
{
    int64_t N = W->N;
    double *ut = (double *)malloc(sizeof(double) * (size_t)N);
    double *ub = (double *)malloc(sizeof(double) * (size_t)N);
    double *R = (double *)malloc(sizeof(double) * (size_t)N);
    int rc = -1;
    if (ut && ub && R && orc_linsys(W, u, ut, 0, NULL) == 0 && eval_R(W, u, ut, ub, R) == 0) {
        for (int64_t i = 0; i < N; ++i) {
            if (Tu) Tu[i] = u[i] - R[i];
            if (Ru) Ru[i] = R[i];
        }
        rc = 0;
    }
    free(ut); free(ub); free(R);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* termination (Sec. 4.3)                                                    */
/*                                                                          */
/* sigma_ = psi_ - 2 psi~ + psi; (x_, y_, s_) = (chi_, psi_, sigma_)/tau_.  */
/* pr, dr, gap as printed.  Reading taken for the certificates (the printed */
/* ratios are negative whenever they apply): ic = ||b|| ||A^T psi_|| /      */
/* (-<b, psi_>), uc = ||c|| ||A chi_ + sigma_|| / (-<c, chi_>), evaluated on */
/* the unscaled vectors.  Order: solved, infeasible, unbounded.             */
/* ------------------------------------------------------------------------ */
int orc_termination(orc_work *W, const double *u, const double *ut, const double *ub, double eps,
                    orc_info *info)
{
    const orc_problem *P = &W->P;
    int32_t n = P->n, m = P->m;
    int64_t N = W->N;
    const double *chib = ub, *psib = ub + n;
    double taub = ub[N - 1];
    double *sig = (double *)malloc(sizeof(double) * (size_t)m);
    double *Ax = (double *)malloc(sizeof(double) * (size_t)m);
    double *ATy = (double *)malloc(sizeof(double) * (size_t)n);
    double *xb = (double *)malloc(sizeof(double) * (size_t)n);
    double *yb = (double *)malloc(sizeof(double) * (size_t)m);
    double *sb = (double *)malloc(sizeof(double) * (size_t)m);
    if (!sig || !Ax || !ATy || !xb || !yb || !sb) {
        free(sig); free(Ax); free(ATy); free(xb); free(yb); free(sb);
        return ORC_NUMERICAL;
    }
    for (int32_t i = 0; i < m; ++i) sig[i] = psib[i] - 2.0 * ut[n + i] + u[n + i];
    double nb = vnorm(P->b, m), nc = vnorm(P->c, n);
    int status = 0;
    info->pr = info->dr = info->gap = INFINITY;
    if (taub > 0.0) {
        for (int32_t j = 0; j < n; ++j) xb[j] = chib[j] / taub;
        for (int32_t i = 0; i < m; ++i) { yb[i] = psib[i] / taub; sb[i] = sig[i] / taub; }
        A_mul(P, xb, Ax);
        AT_mul(P, yb, ATy);
        double s = 0.0;
        for (int32_t i = 0; i < m; ++i) { double e = Ax[i] + sb[i] - P->b[i]; s += e * e; }
        info->pr = sqrt(s) / (1.0 + nb);
        s = 0.0;
        for (int32_t j = 0; j < n; ++j) { double e = ATy[j] + P->c[j]; s += e * e; }
        info->dr = sqrt(s) / (1.0 + nc);
        double cx = vdot(P->c, xb, n), by = vdot(P->b, yb, m);
        info->gap = fabs(cx + by) / (1.0 + fabs(cx) + fabs(by));
        info->pobj = cx;
        info->dobj = -by;
        if (info->pr <= eps && info->dr <= eps && info->gap <= eps) status = ORC_SOLVED;
    }
    /* certificates on unscaled vectors */
    double bpsi = vdot(P->b, psib, m);
    double cchi = vdot(P->c, chib, n);
    AT_mul(P, psib, ATy);
    A_mul(P, chib, Ax);
    info->ic = INFINITY;
    info->uc = INFINITY;
    if (bpsi < 0.0) info->ic = nb * vnorm(ATy, n) / (-bpsi);
    if (cchi < 0.0) {
        double s = 0.0;
        for (int32_t i = 0; i < m; ++i) { double e = Ax[i] + sig[i]; s += e * e; }
        info->uc = nc * sqrt(s) / (-cchi);
    }
    if (!status) {
        if (info->ic < eps) status = ORC_INFEASIBLE;
        else if (info->uc < eps) status = ORC_UNBOUNDED;
    }
    free(sig); free(Ax); free(ATy); free(xb); free(yb); free(sb);
    return status;
}

/* ------------------------------------------------------------------------ */
/* quasi-Newton directions (Sec. 4.4)                                       */
/* ------------------------------------------------------------------------ */
struct orc_dir {
    int32_t kind, mem, count;
    int64_t N, inserted;
    double thetabar, aa_reg;
    double *Z, *Zt; /* mem x N each: z^i and z~^i (RB) or z^i and xi^i (AA) */
    double *v;      /* N scratch */
    double *Q, *R;  /* AA_QR: Q (mem x N, orthonormal columns), R (mem x mem, row-major,
                       upper triangular), Xi_window = Q R with the pairs oldest first */
};

orc_dir *orc_dir_new(int32_t kind, int64_t N, int32_t mem, double thetabar, double aa_reg)
{
    orc_dir *D = (orc_dir *)calloc(1, sizeof(orc_dir));
    if (!D) return NULL;
    D->kind = kind; D->mem = mem < 0 ? 0 : mem; D->N = N;
    if (kind == ORC_DIR_AA_QR && D->mem > 64) D->mem = 64; /* the QR variant keeps at most 64 pairs */
    D->thetabar = thetabar; D->aa_reg = aa_reg;
    size_t cnt = (size_t)(D->mem > 0 ? D->mem : 1) * (size_t)N;
    D->Z = (double *)calloc(cnt, sizeof(double));
    D->Zt = (double *)calloc(cnt, sizeof(double));
    D->v = (double *)calloc((size_t)N, sizeof(double));
    D->Q = (double *)calloc(cnt, sizeof(double));
    D->R = (double *)calloc((size_t)(D->mem > 0 ? D->mem : 1) * (D->mem > 0 ? D->mem : 1), sizeof(double));
    if (!D->Z || !D->Zt || !D->v || !D->Q || !D->R) { orc_dir_free(D); return NULL; }
    return D;
}
void orc_dir_free(orc_dir *D)
{
    if (!D) return;
    free(D->Z); free(D->Zt); free(D->v); free(D->Q); free(D->R); free(D);
}

/* Anderson's acceleration with the least-squares problem min ||Xi t - Ru|| of
 * Sec. 4.4 solved through Xi = Q R, kept up to date as the window moves:
 *  - the oldest pair leaves: R loses its first column, which leaves it upper
 *    Hessenberg; Givens rotations on rows (j, j+1), j = 0..k-2, restore the
 *    triangle and the same rotations combine the columns of Q;
 *  - a new pair xi enters: two rounds of classical Gram-Schmidt against Q
 *    give the new column of R and, normalised, the new column of Q (a pair
 *    whose remainder is below 1e-14 ||xi|| is rank deficient and not stored);
 *  - t solves R t = Q^T Ru by back substitution, d = -Ru - (Z - Xi) t.
 * The columns (Z, Xi, Q) are kept oldest first. */
static void aa_qr_drop_oldest(orc_dir *D)
{
    int64_t N = D->N;
    int32_t k = D->count, m = D->mem;
    double *R = D->R;
    /* R[:, 1:] is k x (k-1) upper Hessenberg */
    for (int32_t j = 0; j + 1 < k; ++j) {
        double a = R[j * m + j + 1], b = R[(j + 1) * m + j + 1];
        double h = hypot(a, b);
        double c = h > 0.0 ? a / h : 1.0, s = h > 0.0 ? b / h : 0.0;
        for (int32_t col = j + 1; col < k; ++col) {
            double x = R[j * m + col], y = R[(j + 1) * m + col];
            R[j * m + col] = c * x + s * y;
            R[(j + 1) * m + col] = -s * x + c * y;
        }
        double *qa = D->Q + (size_t)j * N, *qb = D->Q + (size_t)(j + 1) * N;
        for (int64_t i = 0; i < N; ++i) {
            double x = qa[i], y = qb[i];
            qa[i] = c * x + s * y;
            qb[i] = -s * x + c * y;
        }
    }
    /* shift R's columns left by one (rows 0..k-2) and the windows of Z, Xi */
    for (int32_t r = 0; r + 1 < k; ++r)
        for (int32_t col = 0; col + 1 < k; ++col) R[r * m + col] = col >= r ? R[r * m + col + 1] : 0.0;
    for (int32_t col = 0; col < k; ++col) R[(k - 1) * m + col] = 0.0;
    memmove(D->Z, D->Z + N, sizeof(double) * (size_t)(k - 1) * N);
    memmove(D->Zt, D->Zt + N, sizeof(double) * (size_t)(k - 1) * N);
    D->count = k - 1;
}

static void aa_qr_append(orc_dir *D, const double *z, const double *xi)
{
    int64_t N = D->N;
    int32_t k = D->count, m = D->mem;
    double *w = D->v;
    memcpy(w, xi, sizeof(double) * (size_t)N);
    double nxi = vnorm(xi, N);
    double rcol[64];
    for (int32_t j = 0; j < k; ++j) rcol[j] = 0.0;
    for (int round = 0; round < 2; ++round) {
        double h[64];
        for (int32_t j = 0; j < k; ++j) h[j] = vdot(D->Q + (size_t)j * N, w, N);
        for (int32_t j = 0; j < k; ++j) {
            const double *qj = D->Q + (size_t)j * N;
            for (int64_t i = 0; i < N; ++i) w[i] -= h[j] * qj[i];
            rcol[j] += h[j];
        }
    }
    double rkk = vnorm(w, N);
    if (!(rkk > 1e-14 * nxi)) return; /* rank deficient: the pair is not stored */
    for (int32_t j = 0; j < k; ++j) D->R[j * m + k] = rcol[j];
    D->R[k * m + k] = rkk;
    double *qk = D->Q + (size_t)k * N;
    for (int64_t i = 0; i < N; ++i) qk[i] = w[i] / rkk;
    memcpy(D->Z + (size_t)k * N, z, sizeof(double) * (size_t)N);
    memcpy(D->Zt + (size_t)k * N, xi, sizeof(double) * (size_t)N);
    D->count = k + 1;
}

static void aa_qr_direction(orc_dir *D, const double *r, double *d)
{
    int64_t N = D->N;
    int32_t k = D->count, m = D->mem;
    for (int64_t i = 0; i < N; ++i) d[i] = -r[i];
    if (k == 0) return;
    double t[64];
    for (int32_t j = 0; j < k; ++j) t[j] = vdot(D->Q + (size_t)j * N, r, N);
    for (int32_t j = k - 1; j >= 0; --j) {
        double e = t[j];
        for (int32_t p = j + 1; p < k; ++p) e -= D->R[j * m + p] * t[p];
        t[j] = e / D->R[j * m + j];
    }
    for (int32_t j = 0; j < k; ++j) {
        const double *zj = D->Z + (size_t)j * N, *xj = D->Zt + (size_t)j * N;
        for (int64_t i = 0; i < N; ++i) d[i] -= t[j] * (zj[i] - xj[i]);
    }
}
int32_t orc_dir_count(const orc_dir *D) { return D ? D->count : 0; }

/* Algorithm 2 (modified restarted Broyden).  Readings taken: m' is the number
 * of stored pairs; the loop runs over the stored pairs in insertion order;
 * when m' = mem the buffers are emptied and the current pair is not stored;
 * the denominator of z~ is <z, H xi~> (the printed <s, .> is read as <z, .>);
 * sgn(0) = 1. */
static void rb_direction(orc_dir *D, const double *r, const double *z, const double *xi, double *d)
{
    int64_t N = D->N;
    double *zt = D->v;
    for (int64_t i = 0; i < N; ++i) { d[i] = -r[i]; zt[i] = xi[i]; }
    for (int32_t k = 0; k < D->count; ++k) {
        const double *zk = D->Z + (size_t)k * N, *ztk = D->Zt + (size_t)k * N;
        double a = vdot(zk, zt, N);
        double b = vdot(zk, d, N);
        for (int64_t i = 0; i < N; ++i) { zt[i] += a * ztk[i]; d[i] += b * ztk[i]; }
    }
    double nz2 = vdot(z, z, N);
    double gamma = vdot(zt, z, N) / nz2;
    double sg = gamma >= 0.0 ? 1.0 : -1.0;
    double theta = fabs(gamma) >= D->thetabar ? 1.0 : (1.0 - sg * D->thetabar) / (1.0 - gamma);
    for (int64_t i = 0; i < N; ++i) zt[i] = (1.0 - theta) * z[i] + theta * zt[i];
    double den = vdot(z, zt, N);
    for (int64_t i = 0; i < N; ++i) zt[i] = (z[i] - zt[i]) / den;
    double b = vdot(z, d, N);
    for (int64_t i = 0; i < N; ++i) d[i] += b * zt[i];
    if (D->count == D->mem) {
        D->count = 0;
    } else {
        memcpy(D->Z + (size_t)D->count * N, z, sizeof(double) * (size_t)N);
        memcpy(D->Zt + (size_t)D->count * N, zt, sizeof(double) * (size_t)N);
        D->count++;
    }
}

/* Cholesky solve of a small SPD system (k <= mem), in place; returns 0 on success */
static int small_chol_solve(int32_t k, double *G, double *t)
{
    for (int32_t j = 0; j < k; ++j) {
        double s = G[j * k + j];
        for (int32_t p = 0; p < j; ++p) s -= G[j * k + p] * G[j * k + p];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        G[j * k + j] = ljj;
        for (int32_t i = j + 1; i < k; ++i) {
            double e = G[i * k + j];
            for (int32_t p = 0; p < j; ++p) e -= G[i * k + p] * G[j * k + p];
            G[i * k + j] = e / ljj;
        }
    }
    for (int32_t i = 0; i < k; ++i) {
        double e = t[i];
        for (int32_t p = 0; p < i; ++p) e -= G[i * k + p] * t[p];
        t[i] = e / G[i * k + i];
    }
    for (int32_t i = k - 1; i >= 0; --i) {
        double e = t[i];
        for (int32_t p = i + 1; p < k; ++p) e -= G[p * k + i] * t[p];
        t[i] = e / G[i * k + i];
    }
    return 0;
}

/* Anderson's acceleration: d = -Ru - (Z - Xi) t, t = argmin ||Xi t - Ru||.
 * Readings taken: the buffers are a ring of the last mem pairs (slot =
 * insertion count mod mem, columns used in slot order); the least-squares
 * problem is solved by the normal equations with a Tikhonov term
 * aa_reg * trace(Xi^T Xi) / k, raised tenfold (up to 8 times) if Cholesky
 * fails; if it still fails, d = -Ru. */
static void aa_direction(orc_dir *D, const double *r, double *d)
{
    int64_t N = D->N;
    int32_t k = D->count;
    for (int64_t i = 0; i < N; ++i) d[i] = -r[i];
    if (k == 0) return;
    double *G = (double *)malloc(sizeof(double) * (size_t)k * k);
    double *Gc = (double *)malloc(sizeof(double) * (size_t)k * k);
    double *rhs = (double *)malloc(sizeof(double) * (size_t)k);
    double *t = (double *)malloc(sizeof(double) * (size_t)k);
    if (!G || !Gc || !rhs || !t) { free(G); free(Gc); free(rhs); free(t); return; }
    double tr = 0.0;
    for (int32_t i = 0; i < k; ++i) {
        const double *xi_i = D->Zt + (size_t)i * N;
        for (int32_t j = 0; j <= i; ++j) {
            double g = vdot(xi_i, D->Zt + (size_t)j * N, N);
            G[i * k + j] = g;
            G[j * k + i] = g;
        }
        rhs[i] = vdot(xi_i, r, N);
        tr += G[i * k + i];
    }
    int ok = 0;
    if (tr > 0.0) {
        double reg = D->aa_reg * tr / k;
        for (int attempt = 0; attempt < 8 && !ok; ++attempt, reg *= 10.0) {
            memcpy(Gc, G, sizeof(double) * (size_t)k * k);
            for (int32_t i = 0; i < k; ++i) Gc[i * k + i] += reg;
            memcpy(t, rhs, sizeof(double) * (size_t)k);
            ok = small_chol_solve(k, Gc, t) == 0;
        }
    }
    if (ok) {
        for (int32_t j = 0; j < k; ++j) {
            const double *zj = D->Z + (size_t)j * N, *xj = D->Zt + (size_t)j * N;
            for (int64_t i = 0; i < N; ++i) d[i] -= t[j] * (zj[i] - xj[i]);
        }
    }
    free(G); free(Gc); free(rhs); free(t);
}

int orc_dir_compute(orc_dir *D, const double *Ru, const double *z, const double *xi, int32_t have_pair,
                    double *d)
{
    int64_t N = D->N;
    if (D->kind == ORC_DIR_NONE) {
        for (int64_t i = 0; i < N; ++i) d[i] = 0.0;
        return 0;
    }
    if (have_pair && vdot(z, z, N) == 0.0) have_pair = 0; /* degenerate pair: not used */
    if (D->kind == ORC_DIR_AA_QR) {
        if (have_pair && D->mem > 0) {
            if (D->count == D->mem) aa_qr_drop_oldest(D);
            aa_qr_append(D, z, xi);
        }
        aa_qr_direction(D, Ru, d);
        return 0;
    }
    if (D->kind == ORC_DIR_RB) {
        if (!have_pair) {
            for (int64_t i = 0; i < N; ++i) d[i] = -Ru[i];
            return 0;
        }
        rb_direction(D, Ru, z, xi, d);
        return 0;
    }
    /* AA */
    if (have_pair && D->mem > 0) {
        int32_t slot = (int32_t)(D->inserted % D->mem);
        memcpy(D->Z + (size_t)slot * N, z, sizeof(double) * (size_t)N);
        memcpy(D->Zt + (size_t)slot * N, xi, sizeof(double) * (size_t)N);
        D->inserted++;
        if (D->count < D->mem) D->count++;
    }
    aa_direction(D, Ru, d);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (SuperSCS), with the linearity trick of Sec. 4.2:            */
/*   w~ = u~ + alpha d~ where d~ = (I+Q)^{-1} d is solved once per iteration */
/*                                                                          */
/* Readings taken where the paper is silent:                                */
/*  - u0 = (0, 0, 1) unless a warm start is given;                          */
/*  - q^nu uses the outer iteration index nu;                               */
/*  - backtracking is capped at ls_max halvings; at the cap alpha = 0, so   */
/*    w = u, rho = ||Ru||^2 and K2 is the KM step of Eq. (km);              */
/*  - if ||Rw|| = 0 the point w is a fixed point and is accepted as a K1    */
/*    step (the K2 formula would divide by zero);                           */
/*  - the secant pair handed to the next direction is z = w - u,            */
/*    xi = Rw - Ru with w the last point evaluated (after K0: w = u+d and    */
/*    Rw is the residual of the new iterate);                               */
/*  - after K2 the new u~ is solved directly from the new u;                */
/*  - the termination test runs every check_every iterations on             */
/*    (u, u~, u_) of the current iterate, before the direction.             */
/* ------------------------------------------------------------------------ */
static void write_outputs(orc_work *W, int status, const double *u, const double *ut, const double *ub,
                          double *x, double *y, double *s)
{
    const orc_problem *P = &W->P;
    int32_t n = P->n, m = P->m;
    int64_t N = W->N;
    double taub = ub[N - 1];
    const double *chib = ub, *psib = ub + n;
    for (int32_t i = 0; i < m; ++i) s[i] = psib[i] - 2.0 * ut[n + i] + u[n + i];
    if (status == ORC_INFEASIBLE) {
        double bpsi = vdot(P->b, psib, m);
        for (int32_t i = 0; i < m; ++i) y[i] = psib[i] / (-bpsi);
        for (int32_t j = 0; j < n; ++j) x[j] = NAN;
        for (int32_t i = 0; i < m; ++i) s[i] = NAN;
    } else if (status == ORC_UNBOUNDED) {
        double cchi = vdot(P->c, chib, n);
        for (int32_t j = 0; j < n; ++j) x[j] = chib[j] / (-cchi);
        for (int32_t i = 0; i < m; ++i) { s[i] = s[i] / (-cchi); y[i] = NAN; }
    } else if (taub > 0.0) {
        for (int32_t j = 0; j < n; ++j) x[j] = chib[j] / taub;
        for (int32_t i = 0; i < m; ++i) { y[i] = psib[i] / taub; s[i] = s[i] / taub; }
    } else {
        for (int32_t j = 0; j < n; ++j) x[j] = NAN;
        for (int32_t i = 0; i < m; ++i) { y[i] = NAN; s[i] = NAN; }
    }
}

int orc_solve(orc_work *W, double *x, double *y, double *s, double *u_out, orc_info *info, orc_trace *trace)
{
    const orc_settings *S = &W->S;
    int64_t N = W->N;
    memset(info, 0, sizeof(*info));
    double *buf = (double *)calloc((size_t)N * 12, sizeof(double));
    orc_dir *D = orc_dir_new(S->direction, N, S->mem, S->thetabar, S->aa_reg);
    if (!buf || !D) { free(buf); orc_dir_free(D); info->status = ORC_NUMERICAL; return ORC_NUMERICAL; }
    double *u = buf, *ut = buf + N, *ub = buf + 2 * N, *Ru = buf + 3 * N;
    double *d = buf + 4 * N, *dt = buf + 5 * N, *w = buf + 6 * N, *wt = buf + 7 * N;
    double *wb = buf + 8 * N, *Rw = buf + 9 * N, *zp = buf + 10 * N, *xip = buf + 11 * N;
    int64_t cg0 = W->cg_total;
    if (trace) trace->len = 0;
    /* every solve starts both CG warm starts from zero */
    memset(W->ws[0], 0, sizeof(double) * (size_t)W->P.n);
    memset(W->ws[1], 0, sizeof(double) * (size_t)W->P.n);

    if (S->warm_u) memcpy(u, S->warm_u, sizeof(double) * (size_t)N);
    else u[N - 1] = 1.0;
    orc_linsys(W, u, ut, 0, NULL);
    eval_R(W, u, ut, ub, Ru);
    double nRu = vnorm(Ru, N);
    double eta0 = nRu, r_safe = eta0, eta = eta0;
    W->atol = 0.0;
    int have_pair = 0;
    int status = ORC_MAX_ITERS;
    int check_every = S->check_every > 0 ? S->check_every : 1;
    int nu;
    for (nu = 0; nu < S->max_iters; ++nu) {
        if (!isfinite(nRu)) { status = ORC_NUMERICAL; break; }
        if (nu % check_every == 0) {
            int st = orc_termination(W, u, ut, ub, S->eps, info);
            if (st != 0) { status = st; break; }
        }
        orc_dir_compute(D, Ru, zp, xip, have_pair, d);
        /* reading taken for cg_adapt (not in the paper): inside the loop the CG
         * solves may stop at an absolute residual cg_adapt * ||Ru|| */
        W->atol = S->cg_adapt > 0.0 ? S->cg_adapt * nRu : 0.0;
        orc_linsys(W, d, dt, 1, NULL);
        int step;
        double alpha = 1.0;
        if (trace && trace->len < trace->cap) trace->nRu[trace->len] = nRu;
        if (nRu <= S->c0 * eta) {
            /* K0: blind update u+ = u + d, u~+ = u~ + d~ */
            step = 0;
            eta = nRu;
            for (int64_t i = 0; i < N; ++i) {
                zp[i] = d[i];
                u[i] += d[i];
                ut[i] += dt[i];
            }
            eval_R(W, u, ut, ub, Rw);
            for (int64_t i = 0; i < N; ++i) { xip[i] = Rw[i] - Ru[i]; Ru[i] = Rw[i]; }
            nRu = vnorm(Ru, N);
            info->k0++;
        } else {
            int ls;
            step = -1;
            for (ls = 0; ls <= S->ls_max; ++ls) {
                if (ls == S->ls_max) alpha = 0.0;
                for (int64_t i = 0; i < N; ++i) { w[i] = u[i] + alpha * d[i]; wt[i] = ut[i] + alpha * dt[i]; }
                eval_R(W, w, wt, wb, Rw);
                double nRw = vnorm(Rw, N);
                double rho = 0.0;
                for (int64_t i = 0; i < N; ++i) rho += Rw[i] * (Rw[i] - alpha * d[i]);
                if ((nRu <= r_safe && nRw <= S->c1 * nRu) || nRw == 0.0) {
                    /* K1: u+ = w, reusing w~, w_ and Rw */
                    step = 1;
                    r_safe = nRw + pow(S->q, (double)nu) * eta0;
                    for (int64_t i = 0; i < N; ++i) {
                        zp[i] = alpha * d[i];
                        xip[i] = Rw[i] - Ru[i];
                        u[i] = w[i]; ut[i] = wt[i]; ub[i] = wb[i]; Ru[i] = Rw[i];
                    }
                    nRu = nRw;
                    info->k1++;
                    break;
                } else if (rho >= S->sigma * nRu * nRw) {
                    /* K2: u+ = u - lambda rho / ||Rw||^2 Rw, then a fresh u~ solve */
                    step = 2;
                    double coef = S->lambda * rho / (nRw * nRw);
                    for (int64_t i = 0; i < N; ++i) {
                        zp[i] = alpha * d[i];
                        xip[i] = Rw[i] - Ru[i];
                        u[i] -= coef * Rw[i];
                    }
                    orc_linsys(W, u, ut, 0, NULL);
                    eval_R(W, u, ut, ub, Ru);
                    nRu = vnorm(Ru, N);
                    info->k2++;
                    break;
                }
                alpha *= 0.5;
                info->backtracks++;
            }
        }
        have_pair = 1;
        if (trace && trace->len < trace->cap) {
            trace->step[trace->len] = step;
            trace->alpha[trace->len] = alpha;
            if (trace->ustar && trace->u_dist) {
                double s2 = 0.0;
                for (int64_t i = 0; i < N; ++i) { double e = u[i] - trace->ustar[i]; s2 += e * e; }
                trace->u_dist[trace->len] = sqrt(s2);
            }
            trace->len++;
        }
    }
    if (nu == S->max_iters && status == ORC_MAX_ITERS) {
        /* final test on the last iterate so info reflects where it stopped */
        int st = orc_termination(W, u, ut, ub, S->eps, info);
        if (st != 0) status = st;
    }
    info->iters = nu;
    info->status = status;
    info->nRu = nRu;
    info->cg_iters = W->cg_total - cg0;
    write_outputs(W, status, u, ut, ub, x, y, s);
    if (status == ORC_SOLVED || status == ORC_MAX_ITERS) {
        double cx = vdot(W->P.c, x, W->P.n), by = vdot(W->P.b, y, W->P.m);
        info->pobj = cx;
        info->dobj = -by;
    }
    if (u_out) memcpy(u_out, u, sizeof(double) * (size_t)N);
    W->atol = 0.0;
    free(buf);
    orc_dir_free(D);
    return status;
}
