/*
 * bap_oracle.c -- plain, slow CPU oracle for the nested Monte Carlo continuation estimator of
 * Doan, Gaikwad, Bossy, Baude & Stokes-Rees, "Parallel Pricing Algorithms for Multi-Dimensional
 * Bermudan/American Options using Monte Carlo methods" (INRIA RR-6530, 2008).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the cpu_baseline leg of
 * bench.py may load this code.  It shares no source with the CUDA library (no header, helper,
 * table or constant generator); the two sides agree only on the written random-number contract
 * below, which each implements on its own from the published definitions.
 *
 * Path arithmetic uses the type `real` (double by default; the build also makes a float copy
 * so that exercise decisions can be replayed in single precision).  Every accumulation,
 * discount factor and Newton quantity is double.
 *
 * Random-number contract (both sides implement it separately):
 *   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 *   SC'11): 10 rounds, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments
 *   0x9E3779B9 / 0xBB67AE85.
 *   key = (lo32(seed), hi32(seed) ^ (purpose << 24) ^ m), m = the date being fitted (0 when
 *   pricing).  counter = (path n, item, 4*k + c, 0) for the normals that move a path onto
 *   date k (Philox call c = 0,1,2 gives assets 4c..4c+3); pricing puts hi32(n) in word 1.
 *   Uniforms: v = x >> 9 (23 bits); u1 = (v + 1) * 2^-23 in (0,1], u2 = v * 2^-23 in [0,1).
 *   Box-Muller on words (2p, 2p+1) of a call: z_{4c+2p} = R cos(2 pi u2), z_{4c+2p+1} =
 *   R sin(2 pi u2), R = sqrt(-2 ln u1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real;

#if ORC_REAL_IS_FLOAT
#define R_LOG logf
#define R_EXP expf
#define R_SQRT sqrtf
#define R_COS cosf
#define R_SIN sinf
#define R_TWO_PI 6.28318530717958647692f
#else
#define R_LOG log
#define R_EXP exp
#define R_SQRT sqrt
#define R_COS cos
#define R_SIN sin
#define R_TWO_PI 6.28318530717958647692
#endif

#define ORC_MAXD 16
/* basis size of a cubic in ORC_MAXD - 1 variables: 1 + 15 + 120 + 680 */
#define ORC_MAXBASIS 816

enum { PAY_MAX_CALL = 0, PAY_BASKET_PUT = 1, PAY_GEO_CALL = 2 };
enum { RULE_NONE = 0, RULE_IZ = 1, RULE_CMC = 2 };
enum { ST_OK = 0, ST_NOCONV = 1, ST_NOROOT = 2 };

/* Market model and payoff (Section 2.2 and Section 3.2 of the paper: d correlated GBM assets,
 * constant rate r, dividend yields delta_i, payoff Phi at an exercise date). */
typedef struct {
    int d;
    int n_dates;          /* N_T exercise dates t_1..t_NT */
    int payoff;           /* PAY_* */
    double r, K;
    const double *S0;     /* d */
    const double *sigma;  /* d */
    const double *delta;  /* d */
    const double *w;      /* d: basket weights (arithmetic put, geometric call) */
    const double *t;      /* n_dates + 1, t[0] = 0 */
    const double *L;      /* d*d row-major lower Cholesky factor of the correlation matrix */
} orc_model;

/* A stopping rule for the dates t_1..t_{NT-1}; at t_NT the rule is "exercise iff Phi > 0". */
typedef struct {
    int kind;                     /* RULE_* */
    const unsigned char *fitted;  /* n_dates + 1: nonzero if date k has a fitted rule */
    /* I&Z boundary: x/K = B(y/K), B a polynomial of degree `degree` in the s = d-1 other
     * assets, coefficients ordered [1, y_1..y_s, y_a*y_b (a<=b, lexicographic)] */
    int n_bnd, degree, n_coef;
    const double *coef;           /* (n_dates+1) * n_bnd * n_coef */
    /* CMC boosted stumps: F(S) = sum_s alpha_s h_s(S), h_s = pol_s if feature > thr else -pol_s;
     * features 0..d-1 are the asset prices, feature d is Phi(S) */
    int max_stumps;
    const int *n_stumps;          /* n_dates + 1 */
    const int *feat;              /* (n_dates+1) * max_stumps */
    const double *thr;
    const double *alpha;
    const int *pol;
} orc_rule;

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition (Salmon et al., SC'11).               */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void make_key(uint64_t seed, int purpose, int m, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32) ^ ((uint32_t)purpose << 24) ^ (uint32_t)m;
}

/* d standard normals for one counter prefix (word0, word1, 4*step): Box-Muller on 23-bit
 * uniforms as stated in the header. */
static void normals(const uint32_t key[2], uint32_t w0, uint32_t w1, uint32_t step, int d, real *z)
{
    int n_calls = (d + 3) / 4;
    for (int c = 0; c < n_calls; ++c) {
        uint32_t ctr[4] = {w0, w1, 4u * step + (uint32_t)c, 0u};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        for (int p = 0; p < 2; ++p) {
            int q = 4 * c + 2 * p;
            if (q >= d) break;
            real u1 = (real)((x[2 * p] >> 9) + 1u) * (real)(1.0 / 8388608.0);
            real u2 = (real)(x[2 * p + 1] >> 9) * (real)(1.0 / 8388608.0);
            real R = R_SQRT(-2 * R_LOG(u1));
            z[q] = R * R_COS(R_TWO_PI * u2);
            if (q + 1 < d) z[q + 1] = R * R_SIN(R_TWO_PI * u2);
        }
    }
}

/* Exported for the tests: the normals of one counter prefix, as doubles. */
void orc_normals(uint64_t seed, int purpose, int m, uint32_t w0, uint32_t w1, uint32_t step, int d,
                 double *z_out)
{
    uint32_t key[2];
    real z[ORC_MAXD];
    make_key(seed, purpose, m, key);
    normals(key, w0, w1, step, d, z);
    for (int q = 0; q < d; ++q) z_out[q] = (double)z[q];
}

/* ------------------------------------------------------------------------------------------ */
/* Payoff Phi(S) (Section 2.2: max-call; the basket put and geometric call of the serving mix). */

static double payoff(const orc_model *M, const real *S)
{
    int d = M->d;
    if (M->payoff == PAY_MAX_CALL) {
        real mx = S[0];
        for (int q = 1; q < d; ++q) if (S[q] > mx) mx = S[q];
        double v = (double)mx - M->K;
        return v > 0 ? v : 0;
    } else if (M->payoff == PAY_BASKET_PUT) {
        double b = 0;
        for (int q = 0; q < d; ++q) b += M->w[q] * (double)S[q];
        double v = M->K - b;
        return v > 0 ? v : 0;
    } else {
        double lg = 0;
        for (int q = 0; q < d; ++q) lg += M->w[q] * log((double)S[q]);
        double v = exp(lg) - M->K;
        return v > 0 ? v : 0;
    }
}

/* The asset whose exercise boundary applies at S: for the max-call, the largest asset (first
 * index on ties; one boundary per argmax region, Section 2.2); for the monotone payoffs, asset 0. */
static int rule_pivot(const orc_model *M, const real *S)
{
    if (M->payoff != PAY_MAX_CALL) return 0;
    int best = 0;
    for (int q = 1; q < M->d; ++q) if (S[q] > S[best]) best = q;
    return best;
}

/* d Phi / d S_p * S_p at S (pathwise derivative factor; zero outside the money). */
static double payoff_dlog(const orc_model *M, const real *S, int p)
{
    double phi = payoff(M, S);
    if (phi <= 0) return 0;
    if (M->payoff == PAY_MAX_CALL) return rule_pivot(M, S) == p ? (double)S[p] : 0.0;
    if (M->payoff == PAY_BASKET_PUT) return -M->w[p] * (double)S[p];
    return M->w[p] * (phi + M->K);   /* geometric: w_p * G */
}

/* Polynomial basis of degree <= 3 in s variables, ordered
 * [1, y_a, y_a*y_b (a<=b), y_a*y_b*y_c (a<=b<=c)] (Section 2.2: the boundary is regressed on
 * a quadratic or cubic in the other assets). */
static int basis(int s, int degree, const double *y, double *phi)
{
    int n = 0;
    phi[n++] = 1.0;
    if (degree >= 1) for (int a = 0; a < s; ++a) phi[n++] = y[a];
    if (degree >= 2)
        for (int a = 0; a < s; ++a)
            for (int b = a; b < s; ++b) phi[n++] = y[a] * y[b];
    if (degree >= 3)
        for (int a = 0; a < s; ++a)
            for (int b = a; b < s; ++b)
                for (int c = b; c < s; ++c) phi[n++] = y[a] * y[b] * y[c];
    return n;
}

/* Stopping rule at date k (Section 2.2 for I&Z: exercise when the asset passes the boundary;
 * Section 3.2 for CMC: exercise when F_{t_k}(S) > 0).  Exercise needs Phi > 0; at maturity
 * that alone decides. */
static int exercise(const orc_model *M, const orc_rule *R, int k, const real *S)
{
    double phi = payoff(M, S);
    if (!(phi > 0)) return 0;
    if (k == M->n_dates) return 1;
    if (R->kind == RULE_NONE || !R->fitted[k]) return 0;
    int d = M->d;
    if (R->kind == RULE_IZ) {
        int p = rule_pivot(M, S);
        double y[ORC_MAXD], ph[ORC_MAXBASIS];
        int s = 0;
        for (int q = 0; q < d; ++q) if (q != p) y[s++] = (double)S[q] / M->K;
        int nb = basis(s, R->degree, y, ph);
        const double *c = R->coef + ((size_t)k * R->n_bnd + (R->n_bnd > 1 ? p : 0)) * R->n_coef;
        double B = 0;
        for (int i = 0; i < nb; ++i) B += c[i] * ph[i];
        double xs = (double)S[p] / M->K;
        if (M->payoff == PAY_BASKET_PUT) return xs <= B;
        return xs >= B;
    }
    /* CMC */
    double F = 0;
    int ns = R->n_stumps[k];
    for (int i = 0; i < ns; ++i) {
        size_t o = (size_t)k * R->max_stumps + i;
        int f = R->feat[o];
        double v = f < d ? (double)S[f] : phi;
        double h = v > R->thr[o] ? R->pol[o] : -R->pol[o];
        F += R->alpha[o] * h;
    }
    return F > 0;
}

/* ------------------------------------------------------------------------------------------ */
/* One path from S_{t_m} = start through t_{m+1}..t_NT under the rule (the "small" option price
 * simulations of Section 2.2 and Section 3.2).  Returns the date index of exercise, or
 * n_dates+1 if the path is never exercised (payoff 0).  *disc_phi = exp(-r(t_tau - t_m)) Phi,
 * *disc_dphi = exp(-r(t_tau - t_m)) dPhi/dS_p S_p,tau (divide by the start value for d/dx). */
static int one_path(const orc_model *M, const orc_rule *R, int m, const uint32_t key[2],
                    uint32_t w0, uint32_t w1, const double *start, int pivot,
                    double *disc_phi, double *disc_dphi)
{
    int d = M->d;
    real l[ORC_MAXD], S[ORC_MAXD], z[ORC_MAXD];
    for (int q = 0; q < d; ++q) l[q] = (real)log(start[q]);
    for (int k = m + 1; k <= M->n_dates; ++k) {
        double dt = M->t[k] - M->t[k - 1];
        normals(key, w0, w1, (uint32_t)k, d, z);
        for (int q = 0; q < d; ++q) {
            real wq = 0;
            for (int j = 0; j <= q; ++j) wq += (real)M->L[q * d + j] * z[j];
            real mu = (real)((M->r - M->delta[q] - 0.5 * M->sigma[q] * M->sigma[q]) * dt);
            real sg = (real)(M->sigma[q] * sqrt(dt));
            l[q] = l[q] + mu + sg * wq;
        }
        for (int q = 0; q < d; ++q) S[q] = R_EXP(l[q]);
        if (exercise(M, R, k, S)) {
            double disc = exp(-M->r * (M->t[k] - M->t[m]));
            *disc_phi = disc * payoff(M, S);
            *disc_dphi = pivot >= 0 ? disc * payoff_dlog(M, S, pivot) : 0.0;
            return k;
        }
    }
    *disc_phi = 0;
    *disc_dphi = 0;
    return M->n_dates + 1;
}

/* Nested Monte Carlo continuation estimate for one item: N paths from `start` at t_m.
 * sums[0] = sum of exp(-r(tau-t_m)) Phi, sums[1] = sum of its square, sums[2] = sum of the
 * pathwise derivative with respect to the pivot start value (tau held fixed). */
static void item_sums(const orc_model *M, const orc_rule *R, int m, const uint32_t key[2],
                      uint32_t item, int pivot, const double *start, int64_t N,
                      double sums[3], int64_t *steps)
{
    double s0 = 0, s1 = 0, s2 = 0;
    int64_t st = 0;
    double x = pivot >= 0 ? start[pivot] : 1.0;
    for (int64_t n = 0; n < N; ++n) {
        double a, b;
        int k = one_path(M, R, m, key, (uint32_t)n, item, start, pivot, &a, &b);
        st += (k <= M->n_dates ? k : M->n_dates) - m;
        s0 += a;
        s1 += a * a;
        s2 += b / x;
    }
    sums[0] = s0; sums[1] = s1; sums[2] = s2;
    *steps = st;
}

int orc_continuation(const orc_model *M, const orc_rule *R, int m, int purpose, uint64_t seed,
                     int n_items, const int *item_id, const int *pivot, const double *start,
                     int64_t N, int n_threads, double *sums, int64_t *steps)
{
    if (M->d < 1 || M->d > ORC_MAXD || m < 0 || m >= M->n_dates) return 1;
    uint32_t key[2];
    make_key(seed, purpose, m, key);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < n_items; ++i)
        item_sums(M, R, m, key, (uint32_t)item_id[i], pivot ? pivot[i] : -1,
                  start + (size_t)i * M->d, N, sums + 3 * (size_t)i, steps + i);
    return 0;
}

/* Per-path record for one item: exercise date index (n_dates+1 = never) and the discounted
 * payoff; used to count exercise-decision disagreements path by path. */
int orc_path_trace(const orc_model *M, const orc_rule *R, int m, int purpose, uint64_t seed,
                   int item_id, const double *start, int64_t N, int *tau, double *disc_phi)
{
    if (M->d < 1 || M->d > ORC_MAXD || m < 0 || m >= M->n_dates) return 1;
    uint32_t key[2];
    make_key(seed, purpose, m, key);
    for (int64_t n = 0; n < N; ++n) {
        double b;
        tau[n] = one_path(M, R, m, key, (uint32_t)n, (uint32_t)item_id, start, -1, disc_phi + n, &b);
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* I&Z boundary point: solve Phi(x, y) = C_m(x, y) along the pivot coordinate (Eq. 1, the
 * matched condition P_t(S*) = I(S*); Section 2.3: each point is refined by Newton iterations
 * on N_1 simulated paths).  Safeguarded Newton with a bracket kept from the signs seen, common
 * random numbers across iterates (the counter has no iterate index). */

static double payoff_at(const orc_model *M, const double *start)
{
    real S[ORC_MAXD];
    for (int q = 0; q < M->d; ++q) S[q] = (real)start[q];
    return payoff(M, S);
}

/* I&Z boundary of date k for boundary p at the other assets of S: K B_k(S_{-p}/K) (FP64, the
 * fitted coefficients in basis order). */
static double boundary_value(const orc_model *M, const orc_rule *R, int k, int p, const double *S)
{
    double y[ORC_MAXD], ph[ORC_MAXBASIS];
    int s = 0;
    for (int q = 0; q < M->d; ++q) if (q != p) y[s++] = S[q] / M->K;
    int nb = basis(s, R->degree, y, ph);
    const double *c = R->coef + ((size_t)k * R->n_bnd + (R->n_bnd > 1 ? p : 0)) * R->n_coef;
    double B = 0;
    for (int i = 0; i < nb; ++i) B += c[i] * ph[i];
    return M->K * B;
}

static void newton_item(const orc_model *M, const orc_rule *R, int m, const uint32_t key[2],
                        uint32_t item, int p, const double *start_in, int64_t N,
                        double f_tol, double x_tol, int max_iter, int fixed_point, double fp_eps,
                        int warm_start,
                        double *x_out, int *iters_out, int *status_out, int64_t *steps_out)
{
    int d = M->d;
    double K = M->K;
    double S[ORC_MAXD];
    memcpy(S, start_in, sizeof(double) * d);
    int put_like = M->payoff == PAY_BASKET_PUT;
    double sgn = put_like ? -1.0 : 1.0;
    double lo, hi, x;
    int64_t steps_total = 0;
    *status_out = ST_OK;
    if (M->payoff == PAY_MAX_CALL) {
        double mx = K;
        for (int q = 0; q < d; ++q) if (q != p && start_in[q] > mx) mx = start_in[q];
        lo = mx; hi = INFINITY; x = lo * (1.0 + 1e-3);
    } else if (M->payoff == PAY_GEO_CALL) {
        double lg = log(K);
        for (int q = 0; q < d; ++q) if (q != p) lg -= M->w[q] * log(start_in[q]);
        lo = exp(lg / M->w[p]); hi = INFINITY; x = lo * (1.0 + 1e-3);
    } else {
        double top = K;
        for (int q = 0; q < d; ++q) if (q != p) top -= M->w[q] * start_in[q];
        top /= M->w[p];
        if (!(top > 0)) {
            *x_out = 0; *iters_out = 0; *status_out = ST_NOROOT; *steps_out = 0;
            return;
        }
        lo = 0; hi = top; x = top * (1.0 - 1e-3);
    }
    /* warm start: the later date's fitted boundary at these other assets, when it lies inside
     * the initial bracket (the boundary moves little from one date to the next) */
    if (warm_start && R->kind == RULE_IZ && m + 1 < M->n_dates && R->fitted[m + 1]) {
        double xw = boundary_value(M, R, m + 1, p, start_in);
        if (xw > lo && xw < hi) x = xw;
    }
    double x_max = 1e3 * K, x_min = 1e-6 * K;
    double dx_old = INFINITY, dx = INFINITY;
    int it = 0, done = 0;
    while (it < max_iter) {
        S[p] = x;
        double sums[3];
        int64_t st;
        item_sums(M, R, m, key, item, p, S, N, sums, &st);
        steps_total += st;
        ++it;
        double C = sums[0] / (double)N;
        double dC = sums[2] / (double)N;
        double phi = payoff_at(M, S);
        double f = phi - C;
        if (fixed_point) {
            /* The paper's literal iteration: the next point is the one whose payoff equals the
             * simulated continuation value; stop when it moves by less than eps. */
            double xn;
            if (M->payoff == PAY_MAX_CALL) xn = K + C;
            else if (M->payoff == PAY_GEO_CALL) {
                double lg = log(K + C);
                for (int q = 0; q < d; ++q) if (q != p) lg -= M->w[q] * log(S[q]);
                xn = exp(lg / M->w[p]);
            } else {
                double v = K - C;
                for (int q = 0; q < d; ++q) if (q != p) v -= M->w[q] * S[q];
                xn = v / M->w[p];
                if (xn < 0) xn = 0;
            }
            if (fabs(xn - x) < fp_eps) { x = xn; done = 1; break; }
            x = xn;
            continue;
        }
        if (fabs(f) < f_tol) { done = 1; break; }
        real Sr[ORC_MAXD];
        for (int q = 0; q < d; ++q) Sr[q] = (real)S[q];
        double dphi = payoff_dlog(M, Sr, p) / x;   /* d Phi / d x at the start point */
        double fp = dphi - dC;
        /* g = sgn f increases through the root: keep the bracket lo < root < hi. */
        double g = sgn * f, gp = sgn * fp;
        if (g < 0) lo = x; else hi = x;
        double tol = x_tol * (fabs(x) > 1.0 ? fabs(x) : 1.0);
        if (hi - lo <= tol) { done = 1; break; }
        /* Newton step, unless it leaves the bracket or does not at least halve the step before
         * the last one (the safeguard that breaks 2-cycles across a jump of the simulated
         * function); then bisect, or double x while no upper end is known. */
        double xn = x - g / gp;
        int newton_ok = gp > 0 && xn > lo && xn < hi && fabs(2.0 * g) <= fabs(dx_old * gp);
        if (!newton_ok) xn = isinf(hi) ? 2.0 * x : 0.5 * (lo + hi);
        dx_old = dx;
        dx = xn - x;
        if (xn > x_max) { x = x_max; *status_out = ST_NOROOT; done = 1; break; }
        if (xn < x_min) { x = 0; *status_out = ST_NOROOT; done = 1; break; }
        if (fabs(dx) <= tol) { x = xn; done = 1; break; }
        x = xn;
    }
    if (!done) *status_out = ST_NOCONV;
    *x_out = x;
    *iters_out = it;
    *steps_out = steps_total;
}

int orc_newton(const orc_model *M, const orc_rule *R, int m, int purpose, uint64_t seed,
               int n_items, const int *item_id, const int *pivot, const double *start, int64_t N,
               double f_tol, double x_tol, int max_iter, int fixed_point, double fp_eps,
               int warm_start, int n_threads, double *x_out, int *iters, int *status,
               int64_t *steps)
{
    if (M->d < 1 || M->d > ORC_MAXD || m < 0 || m >= M->n_dates) return 1;
    uint32_t key[2];
    make_key(seed, purpose, m, key);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < n_items; ++i)
        newton_item(M, R, m, key, (uint32_t)item_id[i], pivot[i], start + (size_t)i * M->d, N,
                    f_tol, x_tol, max_iter, fixed_point, fp_eps, warm_start, x_out + i, iters + i,
                    status + i, steps + i);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Final pricing ([mc] phase of Algorithms 1 and 2): N paths from S_0 under the fitted rules;
 * no exercise at t_0; payoff 0 for paths never exercised. */
int orc_price(const orc_model *M, const orc_rule *R, int purpose, uint64_t seed, int64_t N,
              int n_threads, double *sums, int64_t *steps)
{
    if (M->d < 1 || M->d > ORC_MAXD) return 1;
    uint32_t key[2];
    make_key(seed, purpose, 0, key);
    double s0 = 0, s1 = 0;
    int64_t st = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static) reduction(+ : s0, s1, st)
#endif
    for (int64_t n = 0; n < N; ++n) {
        double a, b;
        int k = one_path(M, R, 0, key, (uint32_t)(n & 0xffffffffu), (uint32_t)(n >> 32), M->S0,
                         -1, &a, &b);
        st += k <= M->n_dates ? k : M->n_dates;
        s0 += a;
        s1 += a * a;
    }
    sums[0] = s0; sums[1] = s1; sums[2] = 0;
    *steps = st;
    return 0;
}

/* CMC training points at t_m: independent draws from the law of S_{t_m} given S_0
 * (S = S_0 exp(mu t_m + sqrt(t_m) L z)); counter (j, 0, 4*0 + c, 0) under the TRAIN purpose. */
int orc_train_points(const orc_model *M, int m, int purpose, uint64_t seed, int J, double *X)
{
    if (M->d < 1 || M->d > ORC_MAXD || m < 1 || m > M->n_dates) return 1;
    int d = M->d;
    uint32_t key[2];
    make_key(seed, purpose, m, key);
    double tm = M->t[m];
    for (int j = 0; j < J; ++j) {
        real z[ORC_MAXD];
        normals(key, (uint32_t)j, 0u, 0u, d, z);
        for (int q = 0; q < d; ++q) {
            double wq = 0;
            for (int i = 0; i <= q; ++i) wq += M->L[q * d + i] * (double)z[i];
            double mu = M->r - M->delta[q] - 0.5 * M->sigma[q] * M->sigma[q];
            X[(size_t)j * d + q] = M->S0[q] * exp(mu * tm + M->sigma[q] * sqrt(tm) * wq);
        }
    }
    return 0;
}

/* CMC training points walked back by a Brownian bridge (Section 3.3: the points of date m are
 * simulated backward from those of date m+1).  W is the d-dimensional Brownian motion with
 * covariance rho t that drives log S^q = log S_0^q + mu_q t + sigma_q W^q.  At the last fitted
 * date (Wnext == NULL) W_m = sqrt(t_m) L z, the independent draw; before it, given W at t_{m+1},
 *     W_m = (t_m / t_{m+1}) W_{m+1} + sqrt(t_m (t_{m+1} - t_m) / t_{m+1}) L z,
 * the conditional law of a Brownian motion pinned at 0 at t_0 = 0 and at W_{m+1} at t_{m+1}.
 * z are the same normals as the independent draw of date m (counter (j, 0, c, 0), key of m).
 * Writes W_m (J x d) and the prices X (J x d). */
int orc_train_points_bridge(const orc_model *M, int m, int purpose, uint64_t seed, int J,
                            const double *Wnext, double *W, double *X)
{
    if (M->d < 1 || M->d > ORC_MAXD || m < 1 || m > M->n_dates) return 1;
    if (Wnext && m + 1 > M->n_dates) return 1;
    int d = M->d;
    uint32_t key[2];
    make_key(seed, purpose, m, key);
    double tm = M->t[m];
    double a = 0.0, b = sqrt(tm);
    if (Wnext) {
        double tn = M->t[m + 1];
        a = tm / tn;
        b = sqrt(tm * (tn - tm) / tn);
    }
    for (int j = 0; j < J; ++j) {
        real z[ORC_MAXD];
        normals(key, (uint32_t)j, 0u, 0u, d, z);
        for (int q = 0; q < d; ++q) {
            double lz = 0;
            for (int i = 0; i <= q; ++i) lz += M->L[q * d + i] * (double)z[i];
            double w = b * lz + (Wnext ? a * Wnext[(size_t)j * d + q] : 0.0);
            double mu = M->r - M->delta[q] - 0.5 * M->sigma[q] * M->sigma[q];
            W[(size_t)j * d + q] = w;
            X[(size_t)j * d + q] = M->S0[q] * exp(mu * tm + M->sigma[q] * w);
        }
    }
    return 0;
}

/* Exercise decision of the rule at date k for n given points (tests replay decisions). */
int orc_exercise(const orc_model *M, const orc_rule *R, int k, int n, const double *S, int *out)
{
    for (int i = 0; i < n; ++i) {
        real Sr[ORC_MAXD];
        for (int q = 0; q < M->d; ++q) Sr[q] = (real)S[(size_t)i * M->d + q];
        out[i] = exercise(M, R, k, Sr);
    }
    return 0;
}

int orc_real_bytes(void) { return (int)sizeof(real); }

/* Normals for counters (n, w1, 4*step) with n = 0..count-1 (row n holds d values). */
void orc_normals_bulk(uint64_t seed, int purpose, int m, uint32_t w1, uint32_t step, int d,
                      int64_t count, double *z_out)
{
    uint32_t key[2];
    make_key(seed, purpose, m, key);
    for (int64_t n = 0; n < count; ++n) {
        real z[ORC_MAXD];
        normals(key, (uint32_t)n, w1, step, d, z);
        for (int q = 0; q < d; ++q) z_out[n * d + q] = (double)z[q];
    }
}
