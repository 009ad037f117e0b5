/*
 * dscreen_oracle.c -- plain, slow FP64 CPU oracle for dynamic screening
 * (Bonnefoy, Emiya, Ralaivola, Gribonval, "Dynamic Screening: Accelerating
 * First-Order Algorithms for the Lasso and Group-Lasso", arXiv 1412.4080).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled and called by the test
 * suite, by the smoke check, and by the benchmark's CPU-baseline leg and
 * reference arm.
 * The product (the CUDA library and its Python binding) never links, loads
 * or calls it, and it shares no code, header, table or helper with it.
 *
 * Everything is double precision, single threaded, written as plain loops
 * so that each step can be checked against the paper by eye:
 *
 *   problem         eq. (1): min_x 1/2 ||D x - y||^2 + lambda * Omega(x)
 *   Lasso           eq. (lasso), Omega = ||x||_1, prox = soft threshold (eq. softTh)
 *   Group-Lasso     eq. (group-lasso), Omega = sum_g w_g ||x_g||_2,
 *                   prox = group soft threshold (eq. gr_softTh)
 *   lambda_*        Sec. 2.2.2 (Lasso: ||D^T y||_inf), eq. (gstar) (groups)
 *   updates         Table 1 (ISTA, FISTA, Chambolle-Pock, SpaRSA and TwIST rows;
 *                   backtracking of L for ISTA / FISTA)
 *   general loop    Algorithm 3 (screen after each update, cumulative set)
 *   dual scaling    Lemma 8 (feasible scaled dual point closest to y/lambda)
 *   tests           Lemma 2 (SAFE), Lemma 3 (DST3), Lemma 4 (dynamic Dome),
 *                   Lemma 5 (GSAFE), Lemma 6 (DGST3), Lemma 7 (sphere test)
 *   static variant  Algorithm 1 / Algorithm 4 (test once at theta = -y)
 *   lambda paths    Sec. 5: the sequential test from a previous lambda's dual point
 *
 * The Table 1 recurrences (FISTA's l_t, Chambolle-Pock's steps, schedule and
 * extrapolation) are pinned by iterates worked by hand on a 1 x 1 problem; the
 * constants the paper leaves open (theta_0 = 0, tau_0 = sigma_0 = 0.99 / sqrt(L)) are
 * readings, and those pins fix the oracle to them.
 *
 * Readings of the paper that this file takes (where the text is silent,
 * garbled or specialised):
 *  - theta follows Table 1's sign (theta = D u - y); the clip in Lemma 8
 *    absorbs the sign.  ||theta|| = 0 gives mu = 0.
 *  - the clip of mu uses the correlations of the atoms still active
 *    (Algorithm 5 uses the z of the screened dictionary).
 *  - lambda_* ties and d_*: lowest index attaining the maximum; sign +1
 *    when the correlation is 0.
 *  - atoms of any norm: the Lasso sphere tests are the sphere test of
 *    Lemma 7 with singleton groups, (1 - |d_i^T c|) / ||d_i|| > r, which is
 *    Lemmas 2/3 when ||d_i|| = 1.  DST3 projects y/lambda on the hyperplane
 *    d_*^T theta = 1 (centre y/lambda - psi d_* / ||d_*||^2, offset
 *    psi / ||d_*||, psi = lambda_* / lambda - 1), which is Lemma 3's centre
 *    for a unit d_*.
 *  - Lemma 4 (Dome): the printed inequality compares y^T d_i (the "x^T" and
 *    the stray "l(" are typos), and its piecewise constants are those of the
 *    static test (theta = y, ||y|| = 1).  The dynamic test used here is the
 *    exact maximum of |d^T theta| over the dome {||theta - y/lambda|| <= R,
 *    n^T theta <= 1/||d_*||} for the normalised atom d = d_i/||d_i|| and
 *    normal n = d_* / ||d_*||; it reduces to the printed lemma when theta = y,
 *    ||y|| = 1 and the atoms have unit norm.
 *  - DGST3 radius: Lemma 6's sqrt(||y/lambda - mu theta||^2 -
 *    ||y/lambda - c||^2), clamped at 0 (the appendix prints the operands
 *    of the difference in the opposite order).
 *  - Lemma 8 uses the group of the constraint (the subscript g(i) there is
 *    a typo) and a closed feasible set.
 *  - the duality gap pairs the primal point xbar_t of the iteration with
 *    the dual point v_t = mu_t theta_t built in the same iteration; the
 *    stopping rule is gap <= tol * 1/2 ||y||^2 (= tol * P(0)).
 *  - step size: fixed L >= ||D||_2^2 (power iteration, then * (1 + 1e-6));
 *    the paper's backtracking constants are not given.
 *  - rounding at ties: every test screens only when its margin exceeds
 *    OR_MARGIN = 1e-12 (the paper's strict inequalities, made robust to the
 *    last-bit rounding of double precision).  Without it the atom d_*, which
 *    lies exactly on its own half-space boundary (d_*^T theta <= 1), can be
 *    screened by the Dome / DST3 tests through a rounding error.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_ISTA 0
#define OR_FISTA 1
#define OR_CP 2 /* Chambolle-Pock (Table 1) */
#define OR_SPARSA 3 /* SpaRSA (Table 1): ISTA with a Barzilai-Borwein step */
#define OR_TWIST 4  /* TwIST (Table 1): two-step iterative shrinkage */

/* Constants of the adaptive steps, which the paper leaves to the cited papers (readings):
 * backtracking (Beck-Teboulle) multiplies L by OR_ETA until the quadratic upper model holds;
 * SpaRSA (Wright-Nowak-Figueiredo) accepts a step when F(x_t) <= max of the last OR_SPARSA_M
 * accepted F - OR_SPARSA_SIGMA / 2 alpha ||x_t - x_{t-1}||^2, else multiplies alpha by OR_ETA,
 * and clips its BB step to [OR_BB_MIN, OR_BB_MAX] times L; TwIST (Bioucas-Dias-Figueiredo)
 * replaces a step that increases F by the plain shrinkage step (its monotone variant).  After
 * OR_RETRY_CAP rejections in one iteration the last attempt is kept. */
#define OR_ETA 2.0
#define OR_SPARSA_SIGMA 1e-5
#define OR_SPARSA_M 5
#define OR_BB_MIN 1e-10
#define OR_BB_MAX 1e10
#define OR_RETRY_CAP 40

#define OR_TEST_NONE 0
#define OR_TEST_SAFE 1
#define OR_TEST_DST3 2
#define OR_TEST_DOME 3
#define OR_TEST_GSAFE 4
#define OR_TEST_DGST3 5

/* history columns, one row per iteration */
#define OR_H_ACTIVE 0 /* atoms still active after the screening of iteration t */
#define OR_H_NNZ 1    /* ||xbar_t||_0 */
#define OR_H_R 2      /* R_t = ||y/lambda - mu_t theta_t|| */
#define OR_H_RADIUS 3 /* radius used by the test (R_t or the DST3/DGST3 radius) */
#define OR_H_GAP 4    /* P(xbar_t) - Dual(mu_t theta_t) */
#define OR_H_MU 5     /* mu_t */
#define OR_NH 6

#define OR_MARGIN 1e-12

typedef struct {
    int alg;            /* OR_ISTA / OR_FISTA */
    int test;           /* OR_TEST_* */
    int dynamic;        /* 1: test every iteration (Alg. 3); 0: once, at theta = -y (Alg. 1) */
    int max_iter;       /* iteration cap */
    double tol_gap_rel; /* stop when gap <= tol * 1/2 ||y||^2; 0 runs max_iter iterations */
    double L;           /* step constant; <= 0: power iteration on D^T D, * (1 + 1e-6) */
    double cp_tau;      /* Chambolle-Pock tau_0 and sigma_0 (<= 0: 0.99 / sqrt(L) each, so that */
    double cp_sigma;    /*   tau_0 sigma_0 ||D||^2 < 1) and gamma >= 0 (0: phi_t = 1 throughout) */
    double cp_gamma;
    int step_backtracking; /* ISTA / FISTA: 1 sets L_t by backtracking (Beck-Teboulle) from bt_L0 */
    double bt_L0;          /* first L of the backtracking (<= 0: 1) */
    double twist_xi1;      /* TwIST: lower eigenvalue bound xi_1 of D^T D / L (<= 0: 1e-4) */
    int gap_every;         /* the stopping rule is evaluated every gap_every iterations (<= 1: each) */
} or_options;

typedef struct {
    int iters;
    int n_active;  /* atoms not screened at exit */
    int nnz;
    int status;    /* 0 converged (or max_iter with tol = 0), 1 max_iter reached, -1 bad input */
    double gap;
    double primal;
    double dual;
    double lambda_max;
    double L;
} or_result;

/* ----------------------------------------------------------------- helpers */

static double col_dot(const double* D, int64_t ld, int64_t i, const double* v, int64_t N)
{
    const double* d = D + i * ld;
    double s = 0.0;
    for (int64_t n = 0; n < N; n++) s += d[n] * v[n];
    return s;
}

static double vec_dot(const double* a, const double* b, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Group layout: goff == NULL means the Lasso, i.e. K singleton groups with weight 1. */
static int64_t n_groups(const int64_t* goff, int64_t nG, int64_t K) { return goff ? nG : K; }
static int64_t g_lo(const int64_t* goff, int64_t g) { return goff ? goff[g] : g; }
static int64_t g_hi(const int64_t* goff, int64_t g) { return goff ? goff[g + 1] : g + 1; }
static double g_w(const double* w, int64_t g) { return w ? w[g] : 1.0; }

/* ------------------------------------------------------- lambda_* (Sec. 2.2) */

/* b = D^T y; Lasso: lambda_* = ||D^T y||_inf (Sec. 2.2.2); groups: eq. (gstar),
 * lambda_* = max_g ||D_g^T y|| / w_g.  *star = lowest index attaining it. */
int or_lambda_max(const double* D, int64_t N, int64_t K, int64_t ld, const double* y,
                  const int64_t* goff, const double* w, int64_t nG,
                  double* lambda_max, int64_t* star, double* b)
{
    if (!D || !y || !b || N <= 0 || K <= 0 || ld < N) return -1;
    if (!goff) w = NULL; /* the Lasso: singleton groups of weight 1 */
    for (int64_t i = 0; i < K; i++) b[i] = col_dot(D, ld, i, y, N);
    int64_t G = n_groups(goff, nG, K);
    double best = -1.0;
    int64_t arg = 0;
    for (int64_t g = 0; g < G; g++) {
        double s = 0.0;
        for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) s += b[i] * b[i];
        double v = sqrt(s) / g_w(w, g);
        if (v > best) { best = v; arg = g; }
    }
    *lambda_max = best;
    if (star) *star = arg;
    return 0;
}

/* ---------------------------------------------- spectral norms (step size) */

/* ||D||_2^2 by the power method on D^T D, from the all-ones start vector,
 * until the relative change of the Rayleigh quotient is <= tol. */
double or_spectral_norm_sq(const double* D, int64_t N, int64_t K, int64_t ld, double tol, int max_iter)
{
    double* v = (double*)malloc(sizeof(double) * K);
    double* u = (double*)malloc(sizeof(double) * N);
    for (int64_t i = 0; i < K; i++) v[i] = 1.0 / sqrt((double)K);
    double rq = 0.0;
    for (int it = 0; it < max_iter; it++) {
        for (int64_t n = 0; n < N; n++) u[n] = 0.0;
        for (int64_t i = 0; i < K; i++)
            for (int64_t n = 0; n < N; n++) u[n] += D[i * ld + n] * v[i];
        double rq_new = vec_dot(u, u, N); /* v^T D^T D v with ||v|| = 1 */
        double nv = 0.0;
        for (int64_t i = 0; i < K; i++) { v[i] = col_dot(D, ld, i, u, N); nv += v[i] * v[i]; }
        nv = sqrt(nv);
        if (nv == 0.0) { rq = 0.0; break; }
        for (int64_t i = 0; i < K; i++) v[i] /= nv;
        int done = it > 0 && fabs(rq_new - rq) <= tol * rq_new;
        rq = rq_new;
        if (done) break;
    }
    free(v);
    free(u);
    return rq;
}

/* Largest eigenvalue of the symmetric m x m matrix A (row-major, destroyed)
 * by cyclic Jacobi rotations; returns max diagonal + Frobenius norm of the
 * remaining off-diagonal part, an upper bound (Weyl) that is tight once
 * the sweeps converge. */
static double jacobi_max_eig(double* A, int m)
{
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < m; p++)
            for (int q = 0; q < m; q++)
                if (p != q) off += A[p * m + q] * A[p * m + q];
        if (off == 0.0) break;
        for (int p = 0; p < m - 1; p++) {
            for (int q = p + 1; q < m; q++) {
                double apq = A[p * m + q];
                if (apq == 0.0) continue;
                double app = A[p * m + p], aqq = A[q * m + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < m; k++) { /* A <- A J (columns p, q) */
                    double akp = A[k * m + p], akq = A[k * m + q];
                    A[k * m + p] = c * akp - s * akq;
                    A[k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; k++) { /* A <- J^T A (rows p, q) */
                    double apk = A[p * m + k], aqk = A[q * m + k];
                    A[p * m + k] = c * apk - s * aqk;
                    A[q * m + k] = s * apk + c * aqk;
                }
            }
        }
    }
    double mx = A[0], off = 0.0;
    for (int p = 0; p < m; p++) {
        if (A[p * m + p] > mx) mx = A[p * m + p];
        for (int q = 0; q < m; q++)
            if (p != q) off += A[p * m + q] * A[p * m + q];
    }
    return mx + sqrt(off);
}

/* ||D_g||_2 (spectral norm of the columns c0..c1-1), used by Lemmas 5-7. */
double or_group_spec_norm(const double* D, int64_t N, int64_t ld, int64_t c0, int64_t c1)
{
    int m = (int)(c1 - c0);
    if (m <= 0) return 0.0;
    double* A = (double*)malloc(sizeof(double) * m * m);
    for (int p = 0; p < m; p++)
        for (int q = 0; q < m; q++) A[p * m + q] = vec_dot(D + (c0 + p) * ld, D + (c0 + q) * ld, N);
    double e = jacobi_max_eig(A, m);
    free(A);
    return sqrt(e > 0.0 ? e : 0.0);
}

/* --------------------------------------------------- Lemma 8: dual scaling */

/* mu = [theta^T y / (lambda ||theta||^2)] projected on [-1/m, 1/m], where m is
 * max_i |d_i^T theta| (Lasso) or max_g ||D_g^T theta|| / w_g (groups), i.e.
 * 1/m = s_min of Lemma 8.  ||theta|| = 0 gives 0; m = 0 leaves it unclipped. */
double or_dual_scaling(const double* theta, const double* y, int64_t N, double lambda, double m)
{
    double tt = vec_dot(theta, theta, N);
    if (tt == 0.0) return 0.0;
    double s = vec_dot(theta, y, N) / (lambda * tt);
    if (m > 0.0) {
        double lim = 1.0 / m;
        if (s > lim) s = lim;
        if (s < -lim) s = -lim;
    }
    return s;
}

/* --------------------------------------------------- Lemma 4: dynamic Dome */

/* Maximum of d^T theta over the dome {||theta - c0|| <= R} cap {n^T theta <= off},
 * for unit d and unit n with t = n^T d, dc0 = d^T c0 and psi = n^T c0 - off >= 0
 * (the distance from c0 to the hyperplane, c0 lying outside).  If the unconstrained
 * maximiser c0 + R d satisfies the half-space (t R <= -psi) the value is dc0 + R;
 * otherwise the maximum is on the circle where the sphere meets the hyperplane:
 * dc0 - psi t + sqrt(R^2 - psi^2) sqrt(1 - t^2). */
double or_dome_max(double dc0, double t, double psi, double R)
{
    if (t * R <= -psi) return dc0 + R;
    double rho2 = R * R - psi * psi;
    double s2 = 1.0 - t * t;
    return dc0 - psi * t + sqrt(rho2 > 0 ? rho2 : 0.0) * sqrt(s2 > 0 ? s2 : 0.0);
}

/* ------------------------------------------------------------------ solver */

typedef struct {
    /* per-problem data */
    const double *D, *y;
    int64_t N, K, ld, nG;
    const int64_t* goff;
    const double* w;
    int lasso;
    double lambda, lambda_star;
    int64_t star;
    int test;
    /* per-test data (fixed for the whole solve: Sec. 2.2.4 "D^T c once for all") */
    double* dtc;      /* Lasso: d_i^T c, K entries; groups: ||D_g^T c||, G entries */
    double* nrm;      /* Lasso: ||d_i||; groups: ||D_g||_2 */
    double delta;     /* ||y/lambda - c|| for DST3 / DGST3 (0 for SAFE / GSAFE) */
    /* Dome data (Lasso only) */
    double* b;        /* d_i^T y */
    double* tdome;    /* (d_i / ||d_i||)^T (d_* / ||d_*||) */
    double psi_dome;  /* (lambda_* / lambda - 1) / ||d_*|| */
} or_ctx;

/* Prepare the centre c of the chosen region and D^T c (Lemmas 2, 3, 5, 6). */
static int prepare_test(or_ctx* c, const double* b)
{
    int64_t N = c->N, K = c->K, ld = c->ld;
    int64_t G = n_groups(c->goff, c->nG, K);
    double lam = c->lambda;
    c->delta = 0.0;
    if (c->test == OR_TEST_NONE) return 0;
    if (c->test == OR_TEST_SAFE || c->test == OR_TEST_DST3 || c->test == OR_TEST_DOME) {
        if (!c->lasso) return -1;
    } else if (c->test != OR_TEST_GSAFE && c->test != OR_TEST_DGST3) {
        return -1;
    }
    double* cvec = (double*)malloc(sizeof(double) * N);
    for (int64_t n = 0; n < N; n++) cvec[n] = c->y[n] / lam; /* SAFE / GSAFE centre: y / lambda */
    double psi = c->lambda_star / lam - 1.0;

    if (c->test == OR_TEST_DST3 || c->test == OR_TEST_DOME) {
        /* d_* = argmax over {+-d_i} of d^T y: sign(b_{i*}) d_{i*} (Lemma 3) */
        int64_t is = c->star;
        double sg = b[is] < 0 ? -1.0 : 1.0;
        const double* ds = c->D + is * ld;
        double ns2 = vec_dot(ds, ds, N);
        /* projection of y/lambda on {d_*^T theta = 1}: d_*^T y / lambda - 1 = psi */
        for (int64_t n = 0; n < N; n++) cvec[n] -= psi / ns2 * sg * ds[n];
        c->delta = psi / sqrt(ns2);
        if (c->test == OR_TEST_DOME) {
            c->psi_dome = psi / sqrt(ns2);
            for (int64_t i = 0; i < K; i++) {
                double ni = sqrt(vec_dot(c->D + i * ld, c->D + i * ld, N));
                c->tdome[i] = sg * vec_dot(c->D + i * ld, ds, N) / (ni * sqrt(ns2));
            }
        }
    } else if (c->test == OR_TEST_DGST3) {
        /* n = D_{g*} D_{g*}^T y / lambda_*  (Lemma 6) */
        int64_t gs = c->star;
        double* nv = (double*)calloc(N, sizeof(double));
        for (int64_t i = g_lo(c->goff, gs); i < g_hi(c->goff, gs); i++)
            for (int64_t n = 0; n < N; n++) nv[n] += c->D[i * ld + n] * b[i] / c->lambda_star;
        double nn = vec_dot(nv, nv, N);
        double wg = g_w(c->w, gs);
        double coef = vec_dot(nv, c->y, N) / lam - wg * wg;
        /* c = (I - n n^T/||n||^2) y/lambda + n w^2/||n||^2 = y/lambda - (n^T y/lambda - w^2) n/||n||^2 */
        for (int64_t n = 0; n < N; n++) cvec[n] -= coef * nv[n] / nn;
        c->delta = fabs(coef) / sqrt(nn);
        free(nv);
    }

    if (c->lasso) {
        for (int64_t i = 0; i < K; i++) {
            c->dtc[i] = col_dot(c->D, ld, i, cvec, N);
            c->nrm[i] = sqrt(vec_dot(c->D + i * ld, c->D + i * ld, N));
        }
    } else {
        for (int64_t g = 0; g < G; g++) {
            double s = 0.0;
            for (int64_t i = g_lo(c->goff, g); i < g_hi(c->goff, g); i++) {
                double v = col_dot(c->D, ld, i, cvec, N);
                s += v * v;
            }
            c->dtc[g] = sqrt(s);
            c->nrm[g] = or_group_spec_norm(c->D, N, ld, g_lo(c->goff, g), g_hi(c->goff, g));
        }
    }
    free(cvec);
    return 0;
}

/* Apply the test with dual point theta (whose correlations with the active
 * atoms are z, m = max |z| or max ||z_g||/w_g over active groups).  Marks newly
 * screened groups in scr_group[] with iteration number it.  Returns mu.
 * marg (nullable, G entries) receives each active group's test margin: the
 * quantity the test requires to be positive (sphere tests, Lemma 7:
 * (w_g - ||D_g^T c||) / ||D_g|| - r; Dome, Lemma 4: 1/||d_i|| minus the larger
 * of the two dome maxima), NAN for inactive groups or without a test.  A group
 * is screened when its margin exceeds OR_MARGIN. */
static double screen(or_ctx* c, const double* theta, double m, const char* active_g,
                     int* scr_group, int it, double* R_out, double* rad_out, double* marg)
{
    int64_t N = c->N, K = c->K;
    int64_t G = n_groups(c->goff, c->nG, K);
    double lam = c->lambda;
    /* Lemma 8: mu, v = mu theta; radius R = ||y/lambda - v|| */
    double mu = or_dual_scaling(theta, c->y, N, lam, m);
    double R2 = 0.0;
    for (int64_t n = 0; n < N; n++) {
        double d = c->y[n] / lam - mu * theta[n];
        R2 += d * d;
    }
    double R = sqrt(R2);
    double rad = R;
    if (c->test == OR_TEST_DST3 || c->test == OR_TEST_DGST3) {
        double r2 = R2 - c->delta * c->delta; /* Lemma 3 / Lemma 6 radius */
        rad = sqrt(r2 > 0 ? r2 : 0.0);
    }
    *R_out = R;
    *rad_out = rad;
    if (marg)
        for (int64_t g = 0; g < G; g++) marg[g] = NAN;
    if (c->test == OR_TEST_NONE) return mu;
    for (int64_t g = 0; g < G; g++) {
        if (!active_g[g]) continue;
        double margin;
        if (c->test == OR_TEST_DOME) {
            /* Lemma 4 (dynamic form): max over the dome of |d_i^T theta| < 1 */
            double ni = c->nrm[g];
            double dc0 = c->b[g] / (lam * ni); /* (d_i/||d_i||)^T y / lambda */
            double up = or_dome_max(dc0, c->tdome[g], c->psi_dome, R);
            double lo = or_dome_max(-dc0, -c->tdome[g], c->psi_dome, R);
            margin = 1.0 / ni - (up > lo ? up : lo);
        } else if (c->lasso) {
            /* Lemma 2 / Lemma 3: (1 - |d_i^T c|) / ||d_i|| > r */
            margin = (1.0 - fabs(c->dtc[g])) / c->nrm[g] - rad;
        } else {
            /* Lemma 5 / Lemma 6 via Lemma 7: (w_g - ||D_g^T c||) / ||D_g|| > r */
            margin = (g_w(c->w, g) - c->dtc[g]) / c->nrm[g] - rad;
        }
        if (marg) marg[g] = margin;
        if (margin > OR_MARGIN) scr_group[g] = it;
    }
    return mu;
}

/* Proximal step of Table 1 on group g: x_g = prox_{t Omega}(v_g)
 * (soft threshold eq. softTh, or group soft threshold eq. gr_softTh). */
static void prox_group(const or_ctx* c, int64_t g, const double* v, double t, double* x)
{
    int64_t lo = g_lo(c->goff, g), hi = g_hi(c->goff, g);
    if (c->lasso) {
        double a = fabs(v[lo]) - t;
        x[lo] = a > 0 ? (v[lo] > 0 ? a : -a) : 0.0;
        return;
    }
    double s = 0.0;
    for (int64_t i = lo; i < hi; i++) s += v[i] * v[i];
    double nv = sqrt(s);
    double f = nv > 0 ? (nv - t * g_w(c->w, g)) / nv : 0.0;
    if (f < 0) f = 0.0;
    for (int64_t i = lo; i < hi; i++) x[i] = f * v[i];
}

static double omega(const or_ctx* c, const double* x)
{
    int64_t G = n_groups(c->goff, c->nG, c->K);
    double s = 0.0;
    for (int64_t g = 0; g < G; g++) {
        double q = 0.0;
        for (int64_t i = g_lo(c->goff, g); i < g_hi(c->goff, g); i++) q += x[i] * x[i];
        s += g_w(c->w, g) * sqrt(q);
    }
    return s;
}

/* Table 1 FISTA: l_t = (1 + sqrt(1 + 4 l_{t-1}^2)) / 2; returns the extrapolation
 * coefficient (l_{t-1} - 1) / l_t and advances *lp from l_{t-1} to l_t. */
static double fista_step(double* lp)
{
    double l = *lp;
    double ln = 0.5 * (1.0 + sqrt(1.0 + 4.0 * l * l));
    double beta = (l - 1.0) / ln;
    *lp = ln;
    return beta;
}

/* Dual objective of the gap at the dual point mu theta with R = ||y/lambda - mu theta||:
 * Dual(v) = 1/2 ||y||^2 - lambda^2 / 2 ||v - y/lambda||^2. */
static double dual_objective(double yy, double lambda, double R)
{
    return 0.5 * yy - 0.5 * lambda * lambda * R * R;
}

/* One history row (Sec. 4.1 flops accounting): atoms still active and ||x||_0, with R, the
 * test radius, the gap and mu; also sets res->n_active and res->nnz. */
static void record_iteration(const int64_t* goff, int64_t G, int64_t K, const char* act, const double* x,
                             double R, double rad, double gap, double mu, double* h, or_result* res)
{
    int nact = 0, nnz = 0;
    for (int64_t g = 0; g < G; g++)
        if (act[g]) nact += (int)(g_hi(goff, g) - g_lo(goff, g));
    for (int64_t i = 0; i < K; i++) nnz += x[i] != 0.0;
    if (h) {
        h[OR_H_ACTIVE] = nact;
        h[OR_H_NNZ] = nnz;
        h[OR_H_R] = R;
        h[OR_H_RADIUS] = rad;
        h[OR_H_GAP] = gap;
        h[OR_H_MU] = mu;
    }
    res->n_active = nact;
    res->nnz = nnz;
}

/* Algorithm 3 with the Table 1 rows whose step adapts from one iteration to the next:
 *  - ISTA / FISTA with backtracking (Beck-Teboulle): L_t is the smallest OR_ETA^i L_{t-1}
 *    for which f(xbar_t) <= f(u) + <xbar_t - u, z_t> + L_t/2 ||xbar_t - u||^2, u = ubar_{t-1}
 *    (for the quadratic f: ||D (xbar_t - u)||^2 <= L_t ||xbar_t - u||^2);
 *  - SpaRSA: x_t = prox_{lambda/alpha_t}(xbar_{t-1} - z_t / alpha_t), alpha_1 = L, then the
 *    Barzilai-Borwein value ||D s||^2 / ||s||^2 of the last accepted step s, multiplied by OR_ETA
 *    until F(xbar_t) <= max of the last OR_SPARSA_M accepted F - sigma/2 alpha_t ||s_t||^2;
 *  - TwIST: x_t = (1 - a) x_{t-2} + (a - b) x_{t-1} + b prox_{lambda/L}(x_{t-1} - z_t / L) with
 *    rho = (1 - sqrt(xi_1)) / (1 + sqrt(xi_1)), a = rho^2 + 1, b = 2 a / (1 + xi_1) (the bounds
 *    xi_1 <= eig(D^T D / L) <= 1), and the plain shrinkage step prox_{lambda/L}(x_{t-1} - z_t/L)
 *    for t = 1 and in place of any step that increases F (TwIST's monotone variant).
 * theta_t = D u - y with u = ubar_{t-1} (ISTA, FISTA) or xbar_{t-1} (SpaRSA, TwIST).  The test
 * of iteration t depends on theta_t only, so it is taken first and every acceptance test is
 * evaluated at xbar_t, x_t with the atoms screened at t set to zero.  Returns the number of
 * iterations run; *gap_out, *primal_out, *dual_out as in or_solve_log. */
static int adaptive_loop(or_ctx* c, const or_options* opt, double L, double yy, char* act, int* scr,
                         double* x, double* u, double* theta, double* hist, double* margin_log, int margin_rows,
                         double* gap_out, double* primal_out, double* dual_out, or_result* res)
{
    const double *D = c->D, *y = c->y;
    const int64_t N = c->N, K = c->K, ld = c->ld;
    const int64_t* goff = c->goff;
    const double* w = c->w;
    const int64_t G = n_groups(goff, c->nG, K);
    const double lambda = c->lambda;
    const int sparsa = opt->alg == OR_SPARSA, twist = opt->alg == OR_TWIST, fista = opt->alg == OR_FISTA;
    const int bt = !sparsa && !twist;
    const int ge = opt->gap_every > 1 ? opt->gap_every : 1;
    double* z = (double*)calloc(K, sizeof(double));
    double* v = (double*)calloc(K, sizeof(double));
    double* xn = (double*)calloc(K, sizeof(double));
    double* xb = (double*)calloc(K, sizeof(double));
    double* x2 = (double*)calloc(K, sizeof(double)); /* TwIST: x_{t-2} */
    double* r = (double*)calloc(N, sizeof(double));
    char* kill = (char*)calloc((size_t)G, 1);
    const double xi1 = opt->twist_xi1 > 0 ? opt->twist_xi1 : 1e-4;
    const double rho = (1.0 - sqrt(xi1)) / (1.0 + sqrt(xi1));
    const double ta = rho * rho + 1.0, tb = 2.0 * ta / (1.0 + xi1);
    double Lbt = opt->bt_L0 > 0 ? opt->bt_L0 : 1.0;
    double alpha = L;
    /* F at the starting point, the first entry of SpaRSA's history and TwIST's reference */
    for (int64_t n = 0; n < N; n++) r[n] = -y[n];
    for (int64_t i = 0; i < K; i++)
        if (x[i] != 0.0)
            for (int64_t n = 0; n < N; n++) r[n] += D[i * ld + n] * x[i];
    double Fh[OR_SPARSA_M];
    Fh[0] = 0.5 * vec_dot(r, r, N) + lambda * omega(c, x);
    int nh = 1, hpos = 1;
    double Fprev = Fh[0];
    double l = 1.0; /* FISTA l_0 */
    double gap = INFINITY, primal = 0.0, dual = 0.0;
    int it;
    res->status = 1;
    for (it = 1; it <= opt->max_iter; it++) {
        /* theta_t = D u - y */
        for (int64_t n = 0; n < N; n++) r[n] = -y[n];
        for (int64_t g = 0; g < G; g++) {
            if (!act[g]) continue;
            for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++)
                if (u[i] != 0.0)
                    for (int64_t n = 0; n < N; n++) r[n] += D[i * ld + n] * u[i];
        }
        for (int64_t n = 0; n < N; n++) theta[n] = r[n];
        /* z_t = D_{t-1}^T theta_t and m (Lemma 8) */
        double m = 0.0;
        for (int64_t g = 0; g < G; g++) {
            if (!act[g]) continue;
            double q = 0.0;
            for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) {
                z[i] = col_dot(D, ld, i, theta, N);
                q += z[i] * z[i];
            }
            double val = sqrt(q) / g_w(w, g);
            if (val > m) m = val;
        }
        /* the test of iteration t (Algorithm 3) */
        double R, rad, mu;
        if (opt->dynamic && opt->test != OR_TEST_NONE) {
            mu = screen(c, theta, m, act, scr, it, &R, &rad,
                        margin_log && it < margin_rows ? margin_log + (size_t)it * G : NULL);
        } else {
            int save = c->test;
            c->test = OR_TEST_NONE;
            mu = screen(c, theta, m, act, scr, it, &R, &rad, NULL);
            c->test = save;
        }
        for (int64_t g = 0; g < G; g++) kill[g] = act[g] && scr[g] != 0;
        /* the step, repeated with a larger alpha (L) while its acceptance test fails */
        double Lt = bt ? Lbt : (sparsa ? alpha : L);
        int fallback = 0;
        double F = 0.0, fx = 0.0, dx2 = 0.0;
        for (int tries = 0;; tries++) {
            for (int64_t i = 0; i < K; i++) xb[i] = 0.0;
            for (int64_t g = 0; g < G; g++) {
                if (!act[g]) continue;
                for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) v[i] = (bt ? u[i] : x[i]) - z[i] / Lt;
                prox_group(c, g, v, lambda / Lt, xn);
                for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) {
                    if (twist && it >= 2 && !fallback) xn[i] = (1.0 - ta) * x2[i] + (ta - tb) * x[i] + tb * xn[i];
                    if (!kill[g]) xb[i] = xn[i];
                }
            }
            for (int64_t n = 0; n < N; n++) r[n] = -y[n];
            for (int64_t i = 0; i < K; i++)
                if (xb[i] != 0.0)
                    for (int64_t n = 0; n < N; n++) r[n] += D[i * ld + n] * xb[i];
            fx = 0.5 * vec_dot(r, r, N);
            F = fx + lambda * omega(c, xb);
            dx2 = 0.0;
            for (int64_t i = 0; i < K; i++) dx2 += (xb[i] - x[i]) * (xb[i] - x[i]);
            int ok;
            if (bt) {
                /* the quadratic upper model of f at u: for f = 1/2 ||D x - y||^2,
                 * f(p) = f(u) + <p - u, z> + 1/2 ||D (p - u)||^2 exactly, so the model
                 * f(p) <= f(u) + <p - u, z> + L/2 ||p - u||^2 holds iff ||D (p - u)||^2 <= L ||p - u||^2
                 * (this form has no cancellation near convergence) */
                double sq = 0.0, dq = 0.0;
                for (int64_t i = 0; i < K; i++) sq += (xb[i] - u[i]) * (xb[i] - u[i]);
                for (int64_t n = 0; n < N; n++) {
                    double d = 0.0;
                    for (int64_t i = 0; i < K; i++)
                        if (xb[i] != u[i]) d += D[i * ld + n] * (xb[i] - u[i]);
                    dq += d * d;
                }
                ok = dq <= Lt * sq;
            } else if (sparsa) {
                double Fmax = Fh[0];
                for (int k = 1; k < nh; k++)
                    if (Fh[k] > Fmax) Fmax = Fh[k];
                ok = F <= Fmax - 0.5 * OR_SPARSA_SIGMA * Lt * dx2;
            } else {
                ok = it == 1 || fallback || F <= Fprev;
            }
            if (ok || tries == OR_RETRY_CAP) break;
            if (twist) fallback = 1;
            else Lt *= OR_ETA;
        }
        /* SpaRSA: the Barzilai-Borwein value of the accepted step s = xbar_t - xbar_{t-1} */
        if (sparsa) {
            double ds2 = 0.0;
            for (int64_t n = 0; n < N; n++) {
                double d = 0.0;
                for (int64_t i = 0; i < K; i++)
                    if (xb[i] != x[i]) d += D[i * ld + n] * (xb[i] - x[i]);
                ds2 += d * d;
            }
            alpha = Lt;
            if (dx2 > 0.0) {
                alpha = ds2 / dx2;
                if (alpha < OR_BB_MIN * L) alpha = OR_BB_MIN * L;
                if (alpha > OR_BB_MAX * L) alpha = OR_BB_MAX * L;
            }
        }
        if (bt) Lbt = Lt;
        /* FISTA: l_t and u_t = x_t + ((l_{t-1} - 1) / l_t)(x_t - xbar_{t-1}); the others: u_t = x_t */
        const double beta = fista ? fista_step(&l) : 0.0;
        for (int64_t g = 0; g < G; g++) {
            if (!act[g]) continue;
            for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) {
                if (kill[g]) {
                    x[i] = u[i] = x2[i] = 0.0;
                } else {
                    x2[i] = x[i];
                    u[i] = xn[i] + beta * (xn[i] - x[i]);
                    x[i] = xn[i];
                }
            }
            if (kill[g]) act[g] = 0;
        }
        Fh[hpos] = F;
        hpos = (hpos + 1) % OR_SPARSA_M;
        if (nh < OR_SPARSA_M) nh++;
        Fprev = F;
        /* duality gap P(xbar_t) - Dual(mu_t theta_t) */
        primal = F;
        dual = dual_objective(yy, lambda, R);
        gap = primal - dual;
        record_iteration(goff, G, K, act, x, R, rad, gap, mu, hist ? &hist[(size_t)(it - 1) * OR_NH] : NULL, res);
        if (opt->tol_gap_rel > 0 && it % ge == 0 && gap <= opt->tol_gap_rel * 0.5 * yy) {
            res->status = 0;
            break;
        }
    }
    *gap_out = gap;
    *primal_out = primal;
    *dual_out = dual;
    free(z); free(v); free(xn); free(xb); free(x2); free(r); free(kill);
    return it;
}

/* Solve eq. (1) by Algorithm 3 with the ISTA, FISTA, Chambolle-Pock, SpaRSA or TwIST update
 * of Table 1 (ISTA / FISTA optionally with backtracking; see adaptive_loop).
 * x_out: K coefficients.  scr_iter (nullable): per atom, the iteration at which it
 * was screened (0 = never, -1 = by the static test before the loop).
 * hist (nullable): max_iter rows of OR_NH doubles.
 * theta_out (nullable): N doubles, theta_t of the last iteration run (Table 1's dual
 * variable; left untouched when no iteration runs).
 * margin_log (nullable): margin_rows rows of G doubles (G = groups; the Lasso: K),
 * row 0 the static test of Algorithm 1 and row t the test of iteration t (for
 * t < margin_rows): each group's test margin (see screen()), NAN where the
 * group was not tested. */
int or_solve_log(const double* D, int64_t N, int64_t K, int64_t ld, const double* y, double lambda,
                 const int64_t* goff, const double* w, int64_t nG,
                 const or_options* opt, const double* x0,
                 double* x_out, int* scr_iter, double* hist, double* theta_out, double* margin_log,
                 int margin_rows, or_result* res)
{
    if (!D || !y || !x_out || !opt || !res || N <= 0 || K <= 0 || ld < N || !(lambda > 0)) return -1;
    if (opt->alg < OR_ISTA || opt->alg > OR_TWIST) return -1;
    if (!goff) w = NULL; /* the Lasso: singleton groups of weight 1 */
    if (goff) {
        if (nG <= 0 || goff[0] != 0 || goff[nG] != K) return -1;
        for (int64_t g = 0; g < nG; g++)
            if (goff[g + 1] <= goff[g] || (w && !(w[g] > 0))) return -1;
    }
    memset(res, 0, sizeof(*res));
    or_ctx c;
    memset(&c, 0, sizeof(c));
    c.D = D; c.y = y; c.N = N; c.K = K; c.ld = ld; c.goff = goff; c.w = w; c.nG = nG;
    c.lasso = goff == NULL;
    c.lambda = lambda;
    c.test = opt->test;
    int64_t G = n_groups(goff, nG, K);

    double* b = (double*)malloc(sizeof(double) * K);
    or_lambda_max(D, N, K, ld, y, goff, w, nG, &c.lambda_star, &c.star, b);
    res->lambda_max = c.lambda_star;
    double yy = vec_dot(y, y, N);

    for (int64_t i = 0; i < K; i++) x_out[i] = 0.0;
    if (scr_iter)
        for (int64_t i = 0; i < K; i++) scr_iter[i] = 0;
    if (margin_rows < 1) margin_log = NULL;
    if (margin_log)
        for (int64_t q = 0; q < (int64_t)margin_rows * n_groups(goff, nG, K); q++) margin_log[q] = NAN;
    /* lambda >= lambda_*: x = 0, theta = y/lambda is dual optimal (Sec. 2.2.2, eq. gstar) */
    if (lambda >= c.lambda_star) {
        res->primal = 0.5 * yy;
        res->dual = 0.5 * yy;
        res->gap = 0.0;
        res->n_active = 0;
        free(b);
        return 0;
    }

    double L = opt->L;
    if (!(L > 0)) L = or_spectral_norm_sq(D, N, K, ld, 1e-12, 100000) * (1.0 + 1e-6);
    res->L = L;

    c.dtc = (double*)malloc(sizeof(double) * (size_t)G);
    c.nrm = (double*)malloc(sizeof(double) * (size_t)G);
    c.b = b;
    c.tdome = (double*)malloc(sizeof(double) * (size_t)K);
    if (prepare_test(&c, b) != 0) {
        free(b); free(c.dtc); free(c.nrm); free(c.tdome);
        res->status = -1;
        return -1;
    }

    double* x = (double*)calloc(K, sizeof(double));     /* xbar_{t-1} */
    double* u = (double*)calloc(K, sizeof(double));     /* ubar_{t-1} */
    double* xn = (double*)calloc(K, sizeof(double));    /* x_t */
    double* v = (double*)calloc(K, sizeof(double));
    double* z = (double*)calloc(K, sizeof(double));
    double* theta = (double*)calloc(N, sizeof(double));
    double* r = (double*)calloc(N, sizeof(double));
    char* act = (char*)malloc((size_t)G);
    int* scr = (int*)calloc((size_t)G, sizeof(int));
    for (int64_t g = 0; g < G; g++) act[g] = 1;
    if (x0)
        for (int64_t i = 0; i < K; i++) { x[i] = x0[i]; u[i] = x0[i]; }

    /* Algorithm 1 (static): one test at theta = D*0 - y = -y, before the loop */
    if (!opt->dynamic && opt->test != OR_TEST_NONE) {
        for (int64_t n = 0; n < N; n++) theta[n] = -y[n];
        double m = 0.0;
        for (int64_t g = 0; g < G; g++) {
            double q = 0.0;
            for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) q += b[i] * b[i];
            double val = sqrt(q) / g_w(w, g);
            if (val > m) m = val;
        }
        double R, rad;
        screen(&c, theta, m, act, scr, -1, &R, &rad, margin_log);
        for (int64_t g = 0; g < G; g++)
            if (scr[g]) {
                act[g] = 0;
                for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) { x[i] = 0.0; u[i] = 0.0; }
            }
    }

    int it;
    double gap = INFINITY, primal = 0.0, dual = 0.0;
    if (opt->alg == OR_SPARSA || opt->alg == OR_TWIST ||
        (opt->step_backtracking && (opt->alg == OR_ISTA || opt->alg == OR_FISTA))) {
        it = adaptive_loop(&c, opt, L, yy, act, scr, x, u, theta, hist, margin_log, margin_rows, &gap, &primal,
                           &dual, res);
        goto finish;
    }
    double l = 1.0; /* FISTA l_0 */
    const int cp = opt->alg == OR_CP;
    /* Chambolle-Pock: theta_0 = 0 (dual start), tau_0, sigma_0, gamma (Table 1) */
    double tau = opt->cp_tau > 0 ? opt->cp_tau : 0.99 / sqrt(L);
    double sigma = opt->cp_sigma > 0 ? opt->cp_sigma : 0.99 / sqrt(L);
    const double gamma = opt->cp_gamma > 0 ? opt->cp_gamma : 0.0;
    if (cp)
        for (int64_t n = 0; n < N; n++) theta[n] = 0.0;
    res->status = 1;
    for (it = 1; it <= opt->max_iter; it++) {
        /* Table 1: theta_t = D_{t-1} ubar_{t-1} - y (ISTA, FISTA);
         * Chambolle-Pock: theta_t = (theta_{t-1} + sigma_{t-1} (D_{t-1} ubar_{t-1} - y)) / (1 + sigma_{t-1}) */
        for (int64_t n = 0; n < N; n++) r[n] = -y[n];
        for (int64_t g = 0; g < G; g++) {
            if (!act[g]) continue;
            for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++)
                if (u[i] != 0.0)
                    for (int64_t n = 0; n < N; n++) r[n] += D[i * ld + n] * u[i];
        }
        for (int64_t n = 0; n < N; n++) theta[n] = cp ? (theta[n] + sigma * r[n]) / (1.0 + sigma) : r[n];
        /* z_t = D_{t-1}^T theta_t and the proximal step x_t = prox_{lambda/L}(ubar - z/L)
         * (Chambolle-Pock: x_t = prox_{lambda tau_{t-1}}(xbar_{t-1} - tau_{t-1} z)) */
        double m = 0.0;
        for (int64_t g = 0; g < G; g++) {
            if (!act[g]) continue;
            double q = 0.0;
            for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) {
                z[i] = col_dot(D, ld, i, theta, N);
                q += z[i] * z[i];
                v[i] = cp ? x[i] - tau * z[i] : u[i] - z[i] / L;
            }
            double val = sqrt(q) / g_w(w, g);
            if (val > m) m = val;
            prox_group(&c, g, v, cp ? lambda * tau : lambda / L, xn);
        }
        /* FISTA: l_t and u_t = x_t + ((l_{t-1} - 1) / l_t)(x_t - xbar_{t-1}); ISTA: u_t = x_t;
         * Chambolle-Pock: phi_t = 1 / sqrt(1 + 2 gamma tau_{t-1}), tau_t = phi_t tau_{t-1},
         * sigma_t = sigma_{t-1} / phi_t, u_t = x_t + phi_t (x_t - xbar_{t-1}) */
        double beta = 0.0;
        if (opt->alg == OR_FISTA) {
            beta = fista_step(&l);
        } else if (cp) {
            const double phi = 1.0 / sqrt(1.0 + 2.0 * gamma * tau);
            tau *= phi;
            sigma /= phi;
            beta = phi;
        }
        for (int64_t g = 0; g < G; g++) {
            if (!act[g]) continue;
            for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) {
                double xi = xn[i];
                u[i] = xi + beta * (xi - x[i]);
                x[i] = xi;
            }
        }
        /* screening with theta_t (Algorithm 3 line "I_t <- {i : T_theta_t(i)} u I_{t-1}") */
        double R, rad;
        double mu;
        if (opt->dynamic && opt->test != OR_TEST_NONE) {
            mu = screen(&c, theta, m, act, scr, it, &R, &rad,
                        margin_log && it < margin_rows ? margin_log + (size_t)it * G : NULL);
        } else {
            int save = c.test;
            c.test = OR_TEST_NONE; /* R and mu only, for the gap */
            mu = screen(&c, theta, m, act, scr, it, &R, &rad, NULL);
            c.test = save;
        }
        /* xbar_t, ubar_t: restriction to the atoms still active */
        for (int64_t g = 0; g < G; g++) {
            if (act[g] && scr[g]) {
                act[g] = 0;
                for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) { x[i] = 0.0; u[i] = 0.0; }
            }
        }
        /* duality gap P(xbar_t) - Dual(mu_t theta_t), Dual(v) = 1/2||y||^2 - lambda^2/2 ||v - y/lambda||^2 */
        for (int64_t n = 0; n < N; n++) r[n] = -y[n];
        for (int64_t i = 0; i < K; i++)
            if (x[i] != 0.0)
                for (int64_t n = 0; n < N; n++) r[n] += D[i * ld + n] * x[i];
        primal = 0.5 * vec_dot(r, r, N) + lambda * omega(&c, x);
        dual = dual_objective(yy, lambda, R);
        gap = primal - dual;
        record_iteration(goff, G, K, act, x, R, rad, gap, mu, hist ? hist + (size_t)(it - 1) * OR_NH : NULL, res);
        if (opt->tol_gap_rel > 0 && it % (opt->gap_every > 1 ? opt->gap_every : 1) == 0 &&
            gap <= opt->tol_gap_rel * 0.5 * yy) {
            res->status = 0;
            break;
        }
    }
finish:
    if (it > opt->max_iter) {
        it = opt->max_iter;
        if (!(opt->tol_gap_rel > 0)) res->status = 0;
    }
    res->iters = it;
    res->gap = gap;
    res->primal = primal;
    res->dual = dual;
    for (int64_t i = 0; i < K; i++) x_out[i] = x[i];
    if (theta_out)
        for (int64_t n = 0; n < N; n++) theta_out[n] = theta[n];
    if (scr_iter)
        for (int64_t g = 0; g < G; g++)
            for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) scr_iter[i] = scr[g];

    free(x); free(u); free(xn); free(v); free(z); free(theta); free(r); free(act); free(scr);
    free(b); free(c.dtc); free(c.nrm); free(c.tdome);
    return 0;
}

/* or_solve_log without the margin log. */
int or_solve(const double* D, int64_t N, int64_t K, int64_t ld, const double* y, double lambda,
             const int64_t* goff, const double* w, int64_t nG,
             const or_options* opt, const double* x0,
             double* x_out, int* scr_iter, double* hist, double* theta_out, or_result* res)
{
    return or_solve_log(D, N, K, ld, y, lambda, goff, w, nG, opt, x0, x_out, scr_iter, hist, theta_out, NULL, 0,
                        res);
}

/* Sequential screening along a regularization path (Discussion, Sec. 5): the
 * feasible set of the dual problem, {theta : |d_i^T theta| <= 1} (groups:
 * ||D_g^T theta|| <= w_g), does not depend on lambda, so a dual point scaled
 * into it from any theta -- e.g. the residual D x_k - y of the solution at a
 * previous lambda_k -- yields, by Lemma 8 at the new lambda, a safe region for
 * that lambda.  This applies the chosen test (Lemmas 2-7) once, with the
 * correlations of theta with ALL atoms (the scaling must hold for the whole
 * dictionary, not only for the atoms active at lambda_k).
 * screened (K ints): 1 for the atoms of screened groups, else 0.
 * margin (nullable, G doubles): each group's test margin.  *R_out, *rad_out,
 * *mu_out (nullable): R = ||y/lambda - mu theta||, the test radius, mu.
 * Returns 0, or -1 on bad input (or lambda >= lambda_*, where x = 0 and no
 * test is needed). */
int or_sequential_screen(const double* D, int64_t N, int64_t K, int64_t ld, const double* y, double lambda,
                         const int64_t* goff, const double* w, int64_t nG, int test, const double* theta,
                         int* screened, double* margin, double* R_out, double* rad_out, double* mu_out)
{
    if (!D || !y || !theta || !screened || N <= 0 || K <= 0 || ld < N || !(lambda > 0)) return -1;
    if (!goff) w = NULL;
    or_ctx c;
    memset(&c, 0, sizeof(c));
    c.D = D; c.y = y; c.N = N; c.K = K; c.ld = ld; c.goff = goff; c.w = w; c.nG = nG;
    c.lasso = goff == NULL;
    c.lambda = lambda;
    c.test = test;
    int64_t G = n_groups(goff, nG, K);
    double* b = (double*)malloc(sizeof(double) * K);
    or_lambda_max(D, N, K, ld, y, goff, w, nG, &c.lambda_star, &c.star, b);
    if (lambda >= c.lambda_star) { free(b); return -1; }
    c.dtc = (double*)malloc(sizeof(double) * (size_t)G);
    c.nrm = (double*)malloc(sizeof(double) * (size_t)G);
    c.b = b;
    c.tdome = (double*)malloc(sizeof(double) * (size_t)K);
    char* act = (char*)malloc((size_t)G);
    memset(act, 1, (size_t)G); /* every group is tested */
    int* scr = (int*)calloc((size_t)G, sizeof(int));
    int rc = prepare_test(&c, b);
    if (rc == 0) {
        /* m = max_g ||D_g^T theta|| / w_g over every group */
        double m = 0.0;
        for (int64_t g = 0; g < G; g++) {
            double q = 0.0;
            for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) {
                double z = col_dot(D, ld, i, theta, N);
                q += z * z;
            }
            double val = sqrt(q) / g_w(w, g);
            if (val > m) m = val;
        }
        double R, rad;
        double mu = screen(&c, theta, m, act, scr, 1, &R, &rad, margin);
        for (int64_t g = 0; g < G; g++)
            for (int64_t i = g_lo(goff, g); i < g_hi(goff, g); i++) screened[i] = scr[g] != 0;
        if (R_out) *R_out = R;
        if (rad_out) *rad_out = rad;
        if (mu_out) *mu_out = mu;
    }
    free(b); free(c.dtc); free(c.nrm); free(c.tdome); free(act); free(scr);
    return rc;
}
