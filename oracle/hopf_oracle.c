/*
 * FP64 CPU oracle for the Hopf-formula evaluation of Darbon & Osher,
 * "Algorithms for overcoming the curse of dimensionality for certain
 * Hamilton-Jacobi equations arising in control theory and elsewhere".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never calls it and shares no code with it.
 *
 * Problem (Section 1, eq. 1.2 / Hopf formula; Section 3.1, eq. 3.3):
 *     phi(x,t) = -min_v { J*(v) + t H(v) - <x,v> }
 * with quadratic initial data J(x) = 1/2 (x-c)^T A^{-1} (x-c) - c0, whose
 * Fenchel transform (eq. 1.3) is J*(v) = 1/2 v^T A v + <c,v> + c0, or the
 * initial data of Section 4.4, J = 1/2 |x-c|_1^2 - c0 and 1/2 |x-c|_inf^2 - c0
 * (J* = 1/2 |v|_inf^2 resp. 1/2 |v|_1^2, plus <c,v> + c0), and a positively
 * 1-homogeneous H: l1, weighted l1 (sum w_i |p_i|), l2, l_inf (Section 4.2),
 * sqrt(sum w_i p_i^2) (Section 4.3, diagonal case) or sqrt(<p, M p>) with a
 * symmetric positive definite M (Section 4.3).
 *
 * Algorithm: split Bregman, eq. 3.4(a)-(c), with the paper's start
 * v^0 = d^0 = x (read as y = x - c when a centre is present) and b^0 = 0:
 *   v^{k+1} = argmin J*(v) - <x,v> + lambda/2 |d^k - v - b^k|^2
 *           = (A + lambda I)^{-1} (y + lambda (d^k - b^k))      (prox of a
 *             quadratic form, Section 3.1 / Section 4.1)
 *   d^{k+1} = prox_{(t/lambda) H}(v^{k+1} + b^k)   (shrink_1 / shrink_2,
 *             Section 1 and Section 4.1)
 *   b^{k+1} = b^k + v^{k+1} - d^{k+1}
 * Stopping (Section 4.5): |v^k - v^{k-1}|^2, |d^k - d^{k-1}|^2 and
 * |d^k - v^k|^2 all <= tol ("paper" rule), or, for the relative rule used by
 * the batched GPU solver, |u^k - u^{k-1}|^2 <= tol * max(1, |u^k|^2) for
 * k >= 2, where u^k = v^k + b^{k-1} is the argument of the d-update
 * (u^0 = d^0 + b^0).
 * The returned gradient is d^K (Section 3.1: both (v^k) and (d^k) converge to
 * the minimiser, which is grad_x phi); phi is the objective at d^K.
 *
 * Everything is FP64, unblocked, and written in the paper's order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Initial data: quadratic J with diagonal or dense A, or (Section 4.4)
 * J = 1/2 |x - c|_1^2 - c0 and J = 1/2 |x - c|_inf^2 - c0 (A unused). */
enum { ORC_A_DIAG = 0, ORC_A_DENSE = 1, ORC_J_L1SQ = 2, ORC_J_LINFSQ = 3 };
/* Hamiltonians: l1, weighted l1, l2 (Section 1), l_inf (Section 4.2),
 * H(p) = sqrt(sum_i d_i p_i^2) with d = w (Section 4.3, diagonal case) and
 * H(p) = sqrt(<p, M p>) (Section 4.3).  For ORC_H_ANORM, w holds
 * 2 n^2 + n doubles: M (n x n, row-major), then its eigenvectors P (n x n,
 * row-major, column k the k-th eigenvector) and eigenvalues l (n), with
 * M = P diag(l) P^T; H reads M, the prox reads P and l. */
enum { ORC_H_L1 = 0, ORC_H_WL1 = 1, ORC_H_L2 = 2, ORC_H_LINF = 3, ORC_H_DNORM = 4, ORC_H_ANORM = 5 };
enum { ORC_STOP_PAPER = 0, ORC_STOP_UREL = 1 };

/* One problem instance: A (n diagonal entries or n*n row-major), centre c
 * (n, or NULL for 0), constant c0, Hamiltonian kind and weights w (n, or NULL
 * for all ones), split Bregman lambda, tolerance, iteration cap, stop rule. */
typedef struct {
    int32_t n, a_kind;
    const double *A, *c;
    double c0;
    int32_t h_kind;
    const double *w;
    double lambda, tol;
    int32_t max_iter, stop_rule;
} orc_problem;

/* Per-query results. */
typedef struct {
    double phi;      /* -(J*(d) + t H(d) - <x,d>) at the returned iterate d^K */
    double phi_v;    /* the same objective at v^K (also a lower bound of phi) */
    double dphidt;   /* -H(d^K): the PDE, eq. 1.1a, with grad = d^K */
    int32_t iters;   /* K, the number of v-updates performed */
    int32_t converged;
    double res_paper; /* max of the three paper residuals at K */
    double res_u;     /* |u^K - u^{K-1}|^2 / max(1,|u^K|^2) */
} orc_result;

/* ---- small dense helpers --------------------------------------------- */

/* Cholesky factor L (lower, row-major) of A + lambda I. Returns 0, or -1 when
 * a pivot is not positive (A + lambda I not symmetric positive definite). */
int orc_factor(int32_t n, const double *A, double lambda, double *L)
{
    for (int64_t i = 0; i < (int64_t)n * n; ++i) L[i] = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[(int64_t)i * n + j] + (i == j ? lambda : 0.0);
            for (int k = 0; k < j; ++k) s -= L[(int64_t)i * n + k] * L[(int64_t)j * n + k];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[(int64_t)i * n + i] = sqrt(s);
            } else {
                L[(int64_t)i * n + j] = s / L[(int64_t)j * n + j];
            }
        }
    }
    return 0;
}

/* Solve (A + lambda I) v = r given its Cholesky factor (forward then backward
 * substitution). */
static void chol_solve(int32_t n, const double *L, const double *r, double *v)
{
    for (int i = 0; i < n; ++i) {
        double s = r[i];
        for (int k = 0; k < i; ++k) s -= L[(int64_t)i * n + k] * v[k];
        v[i] = s / L[(int64_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = v[i];
        for (int k = i + 1; k < n; ++k) s -= L[(int64_t)k * n + i] * v[k];
        v[i] = s / L[(int64_t)i * n + i];
    }
}

/* ---- breakpoint algorithms (Sections 4.2 and 4.4) --------------------- */

static int cmp_desc(const void *a, const void *b)
{
    const double x = *(const double *)a, y = *(const double *)b;
    return x < y ? 1 : (x > y ? -1 : 0);
}

/* beta with beta = alpha |shrink_1(z, beta)|_1 (Section 4.4, eq.
 * optimality_beta_l1_2): the breakpoints |z_i| are sorted (decreasing here),
 * the segment on which g(beta) = alpha |shrink_1(z, beta)|_1 - beta changes
 * sign is found, and g, affine there, is interpolated:  on the segment where
 * the k largest |z_i| are active, beta = alpha S_k / (1 + alpha k).  The
 * segment is the first k whose value reaches the next breakpoint (beta_k >=
 * |z|_(k+1)): g is positive at every breakpoint above the root, so for
 * smaller k the value stays below the next breakpoint.  (A two-sided test
 * of beta_k against both ends of its segment can reject both segments that
 * meet at a root lying on a tied breakpoint, by one rounding each.)
 * tmp: n doubles. */
static double l1sq_beta(const double *z, int n, double alpha, double *tmp)
{
    for (int i = 0; i < n; ++i) tmp[i] = fabs(z[i]);
    qsort(tmp, (size_t)n, sizeof(double), cmp_desc);
    double S = 0.0;
    for (int k = 1; k <= n; ++k) {
        S += tmp[k - 1];
        const double beta = alpha * S / (1.0 + alpha * k);
        if (k == n || beta >= tmp[k]) return beta;
    }
    return 0.0;  /* n = 0 */
}

/* exported for the tests */
double orc_l1sq_beta(int32_t n, const double *z, double alpha)
{
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    const double b = l1sq_beta(z, n, alpha, tmp);
    free(tmp);
    return b;
}

/* mu with |shrink_1(z, mu)|_1 = radius, for |z|_1 > radius (Section 4.2:
 * projection on the l1 ball by the Lagrange multiplier of eq.
 * condition_mu_linfty): sorted breakpoints, then on the segment where the k
 * largest |z_i| are active mu = (S_k - radius) / k, the segment being the
 * first k whose value reaches the next breakpoint (as in l1sq_beta).
 * tmp: n doubles. */
static double l1ball_mu(const double *z, int n, double radius, double *tmp)
{
    for (int i = 0; i < n; ++i) tmp[i] = fabs(z[i]);
    qsort(tmp, (size_t)n, sizeof(double), cmp_desc);
    double S = 0.0;
    for (int k = 1; k <= n; ++k) {
        S += tmp[k - 1];
        const double mu = (S - radius) / k;
        if (k == n || mu >= tmp[k]) return mu;
    }
    return 0.0;  /* n = 0 */
}

/* mu > 0 with sum_i s2_i z_i^2 / (s2_i + mu)^2 = 1, for a point outside the
 * ellipsoid {y : sum y_i^2 / s2_i <= 1} (Section 4.3, eq.
 * lagrange_multiplier_equation_ellipsoid): Newton's method on the derivative
 * of F(mu) = sum s2_i z_i^2 / (s2_i + mu) + mu from mu_0 = 0, here run to
 * |mu_{k+1} - mu_k| <= 1e-15 max(1, mu). */
static double ellipsoid_mu(const double *z, const double *s2, int n)
{
    double mu = 0.0;
    for (int it = 0; it < 500; ++it) {
        double f1 = 1.0, f2 = 0.0;  /* F'(mu), F''(mu) */
        for (int i = 0; i < n; ++i) {
            const double q = s2[i] + mu;
            f1 -= s2[i] * z[i] * z[i] / (q * q);
            f2 += 2.0 * s2[i] * z[i] * z[i] / (q * q * q);
        }
        if (!(f2 > 0.0)) break;
        const double dmu = -f1 / f2;
        mu += dmu;
        if (fabs(dmu) <= 1e-15 * (mu > 1.0 ? mu : 1.0)) break;
    }
    return mu;
}

/* v-update, eq. 3.4(a): v = argmin J*(v) - <x, v> + lambda/2 |d - v - b|^2
 * with r = y + lambda (d - b):
 *   quadratic J: v = (A + lambda I)^{-1} r;
 *   J = 1/2 |.-c|_inf^2 (J* = 1/2 |.|_1^2 + <c,.> + c0): v = prox of
 *     (alpha/2)|.|_1^2 at z = r / lambda, alpha = 1 / lambda, i.e.
 *     shrink_1(z, beta) with beta = alpha |shrink_1(z, beta)|_1 (Section 4.4);
 *   J = 1/2 |.-c|_1^2 (J* = 1/2 |.|_inf^2 + ...): v = prox of
 *     (alpha/2)|.|_inf^2 at z, which by Moreau's identity is
 *     z - prox of (1/(2 alpha))|.|_1^2 at z (Section 4.4 writes the identity
 *     for alpha = 1). */
static void v_update(const orc_problem *p, const double *L, const double *r, double *v)
{
    const int n = p->n;
    if (p->a_kind == ORC_A_DIAG) {
        for (int i = 0; i < n; ++i) v[i] = r[i] / (p->A[i] + p->lambda);
    } else if (p->a_kind == ORC_A_DENSE) {
        chol_solve(n, L, r, v);
    } else {
        const double lam = p->lambda;
        double *tmp = (double *)malloc(sizeof(double) * 2 * (size_t)n);
        double *z = tmp + n;
        for (int i = 0; i < n; ++i) z[i] = r[i] / lam;
        const double alpha = 1.0 / lam;
        const double beta = l1sq_beta(z, n, p->a_kind == ORC_J_LINFSQ ? alpha : 1.0 / alpha, tmp);
        for (int i = 0; i < n; ++i) {
            const double sh = z[i] > beta ? z[i] - beta : (z[i] < -beta ? z[i] + beta : 0.0);
            v[i] = p->a_kind == ORC_J_LINFSQ ? sh : z[i] - sh;
        }
        free(tmp);
    }
}

/* H(p): l1, weighted l1, l2, l_inf, or sqrt(sum_i w_i p_i^2) (Section 4.5
 * list of Hamiltonians). */
double orc_H(int32_t h_kind, int32_t n, const double *w, const double *q)
{
    double s = 0.0;
    if (h_kind == ORC_H_LINF) {
        for (int i = 0; i < n; ++i) s = fabs(q[i]) > s ? fabs(q[i]) : s;
        return s;
    }
    if (h_kind == ORC_H_DNORM) {
        for (int i = 0; i < n; ++i) s += w[i] * q[i] * q[i];
        return sqrt(s);
    }
    if (h_kind == ORC_H_ANORM) {
        for (int i = 0; i < n; ++i) {
            double r = 0.0;
            for (int j = 0; j < n; ++j) r += w[(int64_t)i * n + j] * q[j];
            s += q[i] * r;
        }
        return sqrt(s > 0.0 ? s : 0.0);
    }
    if (h_kind == ORC_H_L2) {
        for (int i = 0; i < n; ++i) s += q[i] * q[i];
        return sqrt(s);
    }
    for (int i = 0; i < n; ++i) s += (h_kind == ORC_H_WL1 && w ? w[i] : 1.0) * fabs(q[i]);
    return s;
}

/* prox of tau*H at z, eq. 3.4(b) with alpha = t/lambda:
 *   l1 / weighted l1: shrink_1 per coordinate with threshold tau*w_i,
 *     zero when |z_i| <= threshold (Section 1, definition of shrink_1);
 *   l2: shrink_2(z, tau) = z/|z| max(|z| - tau, 0), and 0 at z = 0. */
void orc_prox(int32_t h_kind, int32_t n, const double *w, double tau, const double *z, double *out)
{
    if (h_kind == ORC_H_ANORM) {
        /* Section 4.3: the dual ball of sqrt(<., M .>) is the ellipsoid
         * {y : <y, M^-1 y> <= 1}, and with M = P diag(l) P^T the projection
         * on it is P times the projection of P^T z on the axis-aligned
         * ellipsoid with weights l; so the prox is the sqrt(sum l p^2) prox
         * in the eigenbasis, rotated back. */
        const double *P = w + (int64_t)n * n, *l = w + 2 * (int64_t)n * n;
        double *zr = (double *)malloc(sizeof(double) * 2 * (size_t)n);
        double *pr = zr + n;
        for (int k = 0; k < n; ++k) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += P[(int64_t)i * n + k] * z[i];
            zr[k] = s;
        }
        orc_prox(ORC_H_DNORM, n, l, tau, zr, pr);
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += P[(int64_t)i * n + k] * pr[k];
            out[i] = s;
        }
        free(zr);
        return;
    }
    if (h_kind == ORC_H_LINF || h_kind == ORC_H_DNORM) {
        /* Moreau's identity: prox of tau |.| = z - projection of z on tau
         * times the dual unit ball (Sections 4.2 and 4.3): the l1 ball for
         * l_inf, the ellipsoid {y : sum y_i^2 / w_i <= 1} for sqrt(sum w p^2) */
        double *tmp = (double *)malloc(sizeof(double) * 2 * (size_t)n);
        if (h_kind == ORC_H_LINF) {
            double l1 = 0.0;
            for (int i = 0; i < n; ++i) l1 += fabs(z[i]);
            if (l1 <= tau) {
                for (int i = 0; i < n; ++i) out[i] = 0.0;
            } else {
                const double mu = l1ball_mu(z, n, tau, tmp);
                for (int i = 0; i < n; ++i) {
                    const double pi = z[i] > mu ? z[i] - mu : (z[i] < -mu ? z[i] + mu : 0.0);
                    out[i] = z[i] - pi;
                }
            }
        } else {
            double *s2 = tmp;
            double inside = 0.0;
            for (int i = 0; i < n; ++i) {
                s2[i] = tau * tau * w[i];
                inside += s2[i] > 0.0 ? z[i] * z[i] / s2[i] : (z[i] != 0.0 ? INFINITY : 0.0);
            }
            if (tau == 0.0) {
                for (int i = 0; i < n; ++i) out[i] = z[i];
            } else if (inside <= 1.0) {
                for (int i = 0; i < n; ++i) out[i] = 0.0;
            } else {
                const double mu = ellipsoid_mu(z, s2, n);
                for (int i = 0; i < n; ++i) out[i] = z[i] * mu / (s2[i] + mu);
            }
        }
        free(tmp);
        return;
    }
    if (h_kind == ORC_H_L2) {
        double nz = 0.0;
        for (int i = 0; i < n; ++i) nz += z[i] * z[i];
        nz = sqrt(nz);
        if (nz == 0.0) {
            for (int i = 0; i < n; ++i) out[i] = 0.0;
            return;
        }
        double m = nz - tau > 0.0 ? nz - tau : 0.0;
        for (int i = 0; i < n; ++i) out[i] = z[i] / nz * m;
        return;
    }
    for (int i = 0; i < n; ++i) {
        double a = tau * (h_kind == ORC_H_WL1 && w ? w[i] : 1.0);
        if (z[i] > a) out[i] = z[i] - a;
        else if (z[i] < -a) out[i] = z[i] + a;
        else out[i] = 0.0;
    }
}

/* 2 J*(v) without the linear part: v^T A v, |v|_inf^2 (J = 1/2|.|_1^2) or
 * |v|_1^2 (J = 1/2|.|_inf^2) */
static double quad_A(const orc_problem *p, const double *v)
{
    double s = 0.0;
    if (p->a_kind == ORC_J_L1SQ) {
        for (int i = 0; i < p->n; ++i) s = fabs(v[i]) > s ? fabs(v[i]) : s;
        return s * s;
    }
    if (p->a_kind == ORC_J_LINFSQ) {
        for (int i = 0; i < p->n; ++i) s += fabs(v[i]);
        return s * s;
    }
    if (p->a_kind == ORC_A_DIAG) {
        for (int i = 0; i < p->n; ++i) s += p->A[i] * v[i] * v[i];
    } else {
        for (int i = 0; i < p->n; ++i) {
            double r = 0.0;
            for (int j = 0; j < p->n; ++j) r += p->A[(int64_t)i * p->n + j] * v[j];
            s += v[i] * r;
        }
    }
    return s;
}

/* -(J*(v) + t H(v) - <x,v>) with J*(v) = 1/2 v^T A v + <c,v> + c0, i.e.
 * <x - c, v> - 1/2 v^T A v - c0 - t H(v): the Hopf objective of eq. 3.3,
 * negated, at the point v. */
double orc_neg_objective(const orc_problem *p, const double *x, double t, const double *v)
{
    double s = 0.0;
    for (int i = 0; i < p->n; ++i) s += (x[i] - (p->c ? p->c[i] : 0.0)) * v[i];
    return s - 0.5 * quad_A(p, v) - p->c0 - t * orc_H(p->h_kind, p->n, p->w, v);
}

/* ---- split Bregman for one query -------------------------------------- */

/* Solve one query.  L is the Cholesky factor from orc_factor (dense A) or
 * NULL (diagonal A).  grad receives d^K (n values). work holds 6n doubles.
 * init (optional, 3n doubles: v^0, d^0, b^0) overrides the paper's start;
 * on return it holds the final (v, d, b), which lets a caller warm-start the
 * next solve (allowed: the iteration converges from any finite start,
 * Section 3.1). */
void orc_solve(const orc_problem *p, const double *L, const double *x, double t,
               double *grad, orc_result *res, double *work, double *init)
{
    const int n = p->n;
    const double lam = p->lambda, tau = t / p->lambda;
    double *y = work, *v = work + n, *d = work + 2 * n, *b = work + 3 * n;
    double *vprev = work + 4 * n, *tmp = work + 5 * n;

    for (int i = 0; i < n; ++i) y[i] = x[i] - (p->c ? p->c[i] : 0.0);
    if (init) {
        for (int i = 0; i < n; ++i) { vprev[i] = init[i]; d[i] = init[n + i]; b[i] = init[2 * n + i]; }
    } else {
        for (int i = 0; i < n; ++i) { vprev[i] = y[i]; d[i] = y[i]; b[i] = 0.0; }
    }
    int k = 0, conv = 0;
    double rp = INFINITY, ru = INFINITY;
    for (k = 1; k <= p->max_iter; ++k) {
        /* eq. 3.4(a): v = (A + lambda I)^{-1} (y + lambda (d - b)) */
        for (int i = 0; i < n; ++i) tmp[i] = y[i] + lam * (d[i] - b[i]);
        v_update(p, L, tmp, v);
        /* u^k = v^k + b^{k-1}; u^{k-1} = v^{k-1} + b^{k-2} = d^{k-1} + b^{k-1} */
        double du = 0.0, un = 0.0;
        for (int i = 0; i < n; ++i) {
            double u = v[i] + b[i];
            double uold = d[i] + b[i];
            tmp[i] = u;
            du += (u - uold) * (u - uold);
            un += u * u;
        }
        /* eq. 3.4(b): d = prox_{tau H}(v + b) */
        double *dn = grad; /* reuse the output buffer as the new d */
        orc_prox(p->h_kind, n, p->w, tau, tmp, dn);
        double r1 = 0.0, r2 = 0.0, r3 = 0.0;
        for (int i = 0; i < n; ++i) {
            r1 += (v[i] - vprev[i]) * (v[i] - vprev[i]);
            r2 += (dn[i] - d[i]) * (dn[i] - d[i]);
            r3 += (dn[i] - v[i]) * (dn[i] - v[i]);
        }
        /* eq. 3.4(c): b = b + v - d */
        for (int i = 0; i < n; ++i) {
            b[i] = b[i] + v[i] - dn[i];
            d[i] = dn[i];
            vprev[i] = v[i];
        }
        rp = r1 > r2 ? r1 : r2;
        rp = rp > r3 ? rp : r3;
        ru = du / (un > 1.0 ? un : 1.0);
        /* The relative rule needs k >= 2: the first step uses the supplied d^0
         * instead of prox(u^0), so u^1 - u^0 is not a fixed-point residual
         * (after a warm start it can vanish while d^0 is far from the answer). */
        if (p->stop_rule == ORC_STOP_PAPER ? (r1 <= p->tol && r2 <= p->tol && r3 <= p->tol)
                                           : (k >= 2 && ru <= p->tol)) {
            conv = 1;
            break;
        }
    }
    if (k > p->max_iter) k = p->max_iter;
    for (int i = 0; i < n; ++i) grad[i] = d[i];
    if (init) {
        for (int i = 0; i < n; ++i) { init[i] = v[i]; init[n + i] = d[i]; init[2 * n + i] = b[i]; }
    }
    res->phi = orc_neg_objective(p, x, t, d);
    res->phi_v = orc_neg_objective(p, x, t, v);
    res->dphidt = -orc_H(p->h_kind, n, p->w, d);
    res->iters = k;
    res->converged = conv;
    res->res_paper = rp;
    res->res_u = ru;
}

/* Batch of queries: x is [batch][n] row-major, t is [batch]; grad is
 * [batch][n]; results are per query.  Queries are independent: each one is
 * its own small problem with no shared state (Section 1; Section 4.5 runs
 * them one per core); with OpenMP they run one per thread.  Returns 0, or -1 if A + lambda I is not SPD. */
int orc_eval_batch(const orc_problem *p, int64_t batch, const double *x, const double *t,
                   double *grad, orc_result *res)
{
    const int n = p->n;
    double *L = NULL;
    if (p->a_kind == ORC_A_DENSE) {
        L = (double *)malloc(sizeof(double) * (size_t)n * n);
        if (!L) return -2;
        if (orc_factor(n, p->A, p->lambda, L) != 0) { free(L); return -1; }
    }
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * 6 * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < batch; ++q)
            orc_solve(p, L, x + q * n, t[q], grad + q * n, res + q, work, NULL);
        free(work);
    }
    free(L);
    return 0;
}

/* Number of threads the OpenMP runtime will use (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- union of initial data (Section 2.2: min over convex initial data) --- */

/* phi = min_i phi_i, where phi_i solves the HJ PDE with initial data J_i; the
 * gradient is that of the minimising part (ties go to the smallest index).
 * parts[i] are independent problems sharing n and H.  argmin[q] receives i*. */
int orc_union_eval(const orc_problem *parts, int32_t K, int64_t batch, const double *x,
                   const double *t, double *phi, double *grad, int32_t *argmin, int32_t *iters)
{
    const int n = parts[0].n;
    double **L = (double **)calloc((size_t)K, sizeof(double *));
    for (int i = 0; i < K; ++i) {
        if (parts[i].a_kind == ORC_A_DENSE) {
            L[i] = (double *)malloc(sizeof(double) * (size_t)n * n);
            if (orc_factor(n, parts[i].A, parts[i].lambda, L[i]) != 0) {
                for (int j = 0; j <= i; ++j) free(L[j]);
                free(L);
                return -1;
            }
        }
    }
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * 6 * (size_t)n);
        double *g = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < batch; ++q) {
            double best = INFINITY;
            int bi = -1, it = 0;
            for (int i = 0; i < K; ++i) {
                orc_result r;
                orc_solve(&parts[i], L[i], x + q * n, t[q], g, &r, work, NULL);
                it += r.iters;
                if (r.phi < best) {
                    best = r.phi;
                    bi = i;
                    memcpy(grad + q * n, g, sizeof(double) * (size_t)n);
                }
            }
            phi[q] = best;
            argmin[q] = bi;
            iters[q] = it;
        }
        free(work);
        free(g);
    }
    for (int i = 0; i < K; ++i) free(L[i]);
    free(L);
    return 0;
}

/* ---- distance and closest point by the level-set route (Section 3.2) ---- */

/* For one part with H = l2: psi(y,s) solves the eikonal equation (3.8) with
 * initial data J_i, and psi(y,s) = 0 exactly when y lies at Euclidean distance
 * s from the set {J_i <= 0}.  Newton's method on s (eq. Newton_zero) uses
 * d psi/ds = -|grad psi| (from the PDE):  s <- s + psi(y,s)/|grad psi(y,s)|.
 * Start s_0 = 0; stop when |s_{l+1} - s_l| <= s_tol * max(1, s), at most
 * max_newton steps.  Each step is one Hopf evaluation by split Bregman,
 * warm-started from the previous step's (v, d, b).  On return: *s_bar and the
 * projection y - s_bar grad psi / |grad psi| (eq. projection_when_s_known).
 * Returns the number of Newton steps, or -1 without convergence. */
int orc_closest_point_one(const orc_problem *p, const double *L, const double *y, double s_tol,
                          int32_t max_newton, double *s_bar, double *proj, int32_t *iters,
                          double *work /* 10n */)
{
    const int n = p->n;
    double *g = work + 6 * n, *state = work + 7 * n;
    double s = 0.0;
    int it = 0, l;
    orc_result r;
    for (int i = 0; i < n; ++i) { state[i] = y[i] - (p->c ? p->c[i] : 0.0); state[n + i] = state[i]; state[2 * n + i] = 0.0; }
    int ok = -1;
    for (l = 0; l < max_newton; ++l) {
        orc_solve(p, L, y, s, g, &r, work, state);
        it += r.iters;
        double gn = 0.0;
        for (int i = 0; i < n; ++i) gn += g[i] * g[i];
        gn = sqrt(gn);
        if (!(gn > 0.0)) break;
        double ds = r.phi / gn;
        s += ds;
        if (fabs(ds) <= s_tol * (s > 1.0 ? s : 1.0)) { ok = l + 1; break; }
    }
    /* gradient at the final s */
    orc_solve(p, L, y, s, g, &r, work, state);
    it += r.iters;
    double gn = 0.0;
    for (int i = 0; i < n; ++i) gn += g[i] * g[i];
    gn = sqrt(gn);
    for (int i = 0; i < n; ++i) proj[i] = y[i] - s * g[i] / gn;
    *s_bar = s;
    *iters = it;
    return ok;
}

/* Union version: distance = min_i s_bar_i (ties to the smallest i), closest
 * point = the projection onto that part (Section 2.2 with Section 3.2). */
int orc_union_closest(const orc_problem *parts, int32_t K, int64_t batch, const double *x,
                      double s_tol, int32_t max_newton, double *dist, double *closest,
                      int32_t *argmin, int32_t *newton_fail)
{
    const int n = parts[0].n;
    double **L = (double **)calloc((size_t)K, sizeof(double *));
    for (int i = 0; i < K; ++i) {
        if (parts[i].a_kind == ORC_A_DENSE) {
            L[i] = (double *)malloc(sizeof(double) * (size_t)n * n);
            if (orc_factor(n, parts[i].A, parts[i].lambda, L[i]) != 0) {
                for (int j = 0; j <= i; ++j) free(L[j]);
                free(L);
                return -1;
            }
        }
    }
    int fails = 0;
#pragma omp parallel reduction(+ : fails)
    {
        double *work = (double *)malloc(sizeof(double) * 10 * (size_t)n);
        double *pr = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < batch; ++q) {
            double best = INFINITY;
            int bi = -1;
            for (int i = 0; i < K; ++i) {
                double sb;
                int32_t it;
                int ok = orc_closest_point_one(&parts[i], L[i], x + q * n, s_tol, max_newton, &sb, pr, &it, work);
                if (ok < 0) fails += 1;
                if (sb < best) {
                    best = sb;
                    bi = i;
                    memcpy(closest + q * n, pr, sizeof(double) * (size_t)n);
                }
            }
            dist[q] = best;
            argmin[q] = bi;
        }
        free(work);
        free(pr);
    }
    for (int i = 0; i < K; ++i) free(L[i]);
    free(L);
    *newton_fail = fails;
    return 0;
}

/* ---- gradients of phi with respect to the data (envelope theorem) ------
 * phi(x,t;A,c,c0,w) = max_v -F(v) with F the Hopf objective of eq. 3.3, so
 * with v* the (unique) minimiser: d/dx = v*, d/dt = -H(v*),
 * d/dA = -1/2 v* v*^T, d/dc = -v*, d/dc0 = -1, d/dw_i = -t |v*_i|.
 * Batched with upstream weights g_q: gA = -1/2 sum_q g_q v*_q v*_q^T (dense) or
 * its diagonal.  gx and gt are per query. */
void orc_backward(int32_t n, int32_t a_kind, int32_t h_kind, const double *w, int64_t batch,
                  const double *g_phi, const double *vstar, const double *t, double *g_x,
                  double *g_t, double *g_A /* n*n or n, may be NULL */)
{
    if (g_A) {
        int64_t m = a_kind == ORC_A_DENSE ? (int64_t)n * n : n;
        for (int64_t i = 0; i < m; ++i) g_A[i] = 0.0;
    }
    for (int64_t q = 0; q < batch; ++q) {
        const double *v = vstar + q * n;
        for (int i = 0; i < n; ++i) g_x[q * n + i] = g_phi[q] * v[i];
        g_t[q] = -g_phi[q] * orc_H(h_kind, n, w, v);
        if (g_A) {
            if (a_kind == ORC_A_DENSE) {
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) g_A[(int64_t)i * n + j] -= 0.5 * g_phi[q] * v[i] * v[j];
            } else {
                for (int i = 0; i < n; ++i) g_A[i] -= 0.5 * g_phi[q] * v[i] * v[i];
            }
        }
    }
    (void)t;
}

/* Gradients with respect to the other parameters of the problem, by the
 * same envelope argument on eq. 3.3 (phi = <x - c, p> - J*_0(p) - c0 - t H(p)
 * at the minimiser p):
 *   d phi / d c    = -p            (J depends on x - c),
 *   d phi / d c0   = -1,
 *   d phi / d w_i  = -t |p_i|                 (H = sum_i w_i |p_i|),
 *                  = -t p_i^2 / (2 H(p))      (H = sqrt(sum_i w_i p_i^2), 0 at p = 0).
 * With upstream weights g_q, summed over the batch: g_c (n), g_c0 (1) and
 * g_w (n, weighted kinds only; may be NULL). */
void orc_backward_params(int32_t n, int32_t h_kind, const double *w, int64_t batch, const double *g_phi,
                         const double *vstar, const double *t, double *g_c, double *g_c0, double *g_w)
{
    for (int i = 0; i < n; ++i) {
        g_c[i] = 0.0;
        if (g_w) g_w[i] = 0.0;
    }
    *g_c0 = 0.0;
    for (int64_t q = 0; q < batch; ++q) {
        const double *v = vstar + q * n;
        *g_c0 -= g_phi[q];
        for (int i = 0; i < n; ++i) g_c[i] -= g_phi[q] * v[i];
        if (g_w && h_kind == ORC_H_WL1) {
            for (int i = 0; i < n; ++i) g_w[i] -= g_phi[q] * t[q] * fabs(v[i]);
        } else if (g_w && h_kind == ORC_H_DNORM) {
            const double H = orc_H(h_kind, n, w, v);
            if (H > 0.0)
                for (int i = 0; i < n; ++i) g_w[i] -= g_phi[q] * t[q] * v[i] * v[i] / (2.0 * H);
        }
    }
}

/* ---- optimal control and terminal point (Section 2, the control remark and
 *      the Hopf-Lax discussion at the end of Section 2.2) ------------------- */

/* For the minimiser p of eq. 3.3 at (x, t), t > 0, the optimality condition
 * 0 in A p + c - x + t dH(p) gives the control as the element of dH(p)
 *     beta = (x - c - A p) / t,
 * which equals grad H(p) wherever H is differentiable (the paper's
 * beta(t) = grad H(grad phi)), and the terminal point of the optimal
 * trajectory, the minimiser of the Hopf-Lax formula, x_T = x - t beta
 * (= c + A p).  At t = 0 the control is taken as 0 and x_T = x.
 * beta and x_T hold batch x n values; grad holds the minimisers. */
void orc_control(const orc_problem *p, int64_t batch, const double *x, const double *t, const double *grad,
                 double *beta, double *x_T)
{
    const int n = p->n;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < batch; ++q) {
        const double *g = grad + q * n;
        if (p->a_kind != ORC_A_DIAG && p->a_kind != ORC_A_DENSE) {
            /* J* is not differentiable there: the control is not defined by
             * this formula */
            for (int i = 0; i < n; ++i) beta[q * n + i] = x_T[q * n + i] = NAN;
            continue;
        }
        for (int i = 0; i < n; ++i) {
            double ap = 0.0;
            if (p->a_kind == ORC_A_DIAG) ap = p->A[i] * g[i];
            else
                for (int j = 0; j < n; ++j) ap += p->A[(int64_t)i * n + j] * g[j];
            const double xi = x[q * n + i];
            const double b = t[q] > 0.0 ? (xi - (p->c ? p->c[i] : 0.0) - ap) / t[q] : 0.0;
            beta[q * n + i] = b;
            x_T[q * n + i] = xi - t[q] * b;
        }
    }
}

/* ---- maximum over Hamiltonians (Section 2.2, the remark on the minimum of
 *      Hamiltonians): for k Hamiltonians H_i and one initial data J,
 *      max_i phi_i solves the HJ equation with Hamiltonian min_i H_i. ------- */

/* parts[i] share n, A, c and c0 and differ in H (kind and weights).  phi[q]
 * = max_i phi_i(x_q, t_q), argmax[q] = the first maximising i, grad = the
 * gradient of that part, iters = the iterations summed over parts. */
int orc_maxH_eval(const orc_problem *parts, int32_t K, int64_t batch, const double *x, const double *t,
                  double *phi, double *grad, int32_t *argmax, int32_t *iters)
{
    const int n = parts[0].n;
    double *L = NULL;
    if (parts[0].a_kind == ORC_A_DENSE) {
        L = (double *)malloc(sizeof(double) * (size_t)n * n);
        if (orc_factor(n, parts[0].A, parts[0].lambda, L) != 0) { free(L); return -1; }
    }
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * 6 * (size_t)n);
        double *g = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < batch; ++q) {
            double best = -INFINITY;
            int bi = -1, it = 0;
            for (int i = 0; i < K; ++i) {
                orc_result r;
                orc_solve(&parts[i], L, x + q * n, t[q], g, &r, work, NULL);
                it += r.iters;
                if (r.phi > best) {
                    best = r.phi;
                    bi = i;
                    memcpy(grad + q * n, g, sizeof(double) * (size_t)n);
                }
            }
            phi[q] = best;
            argmax[q] = bi;
            iters[q] = it;
        }
        free(work);
        free(g);
    }
    free(L);
    return 0;
}
