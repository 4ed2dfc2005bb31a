/*
 * bap.h -- C ABI of the GB300 (sm_103a) nested Monte Carlo Bermudan/American option library.
 *
 * Method: Doan, Gaikwad, Bossy, Baude & Stokes-Rees, "Parallel Pricing Algorithms for
 * Multi-Dimensional Bermudan/American Options using Monte Carlo methods", INRIA RR-6530 (2008):
 *   - Section 2 (Algorithm 1): Ibanez-Zapatero exercise-boundary search.  At every exercise date,
 *     backward in time, boundary points solve the matched condition P_t(S*) = I(S*) (Eq. 1) by
 *     Newton iterations on nested Monte Carlo continuation values; a polynomial boundary is
 *     regressed on the points; the price is a Monte Carlo mean under the fitted boundaries.
 *   - Section 3 (Algorithm 2): Picazo classification Monte Carlo.  Training points are labelled by
 *     the sign of (exercise value - continuation value) and a boosted classifier F_t with
 *     sign F_t = sign beta(t, .) gives the stopping rule tau = min{t_m : F_{t_m}(S) > 0}.
 *
 * Conventions for every call:
 *   - Pointers are HOST pointers unless a parameter says otherwise.  The caller owns every input
 *     array; the library copies what it keeps before the call returns.
 *   - The library owns the handles and all device memory they hold.  Results go to caller-owned
 *     host memory.
 *   - Errors come back as a bap_status; nothing throws or exits across the ABI.  A thread-local
 *     message for the last failure is available from bap_last_error().
 *   - A bap_option is not thread safe; use one thread per option (or serialize).  bap_server is
 *     thread safe for bap_submit and bap_poll.
 *   - Everything runs on the CUDA device current at bap_create, on the option's stream (default:
 *     a stream the library creates; see bap_set_stream).  Calls that return results synchronize
 *     that stream.
 *   - There is no CPU fallback: without a CUDA device every compute call returns BAP_ECUDA.
 */
#ifndef BAP_H
#define BAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BAP_OK = 0,
    BAP_EINVAL = 1,     /* bad argument (message in bap_last_error) */
    BAP_ENOMEM = 2,     /* device or host allocation failed */
    BAP_ECUDA = 3,      /* CUDA error, or no CUDA device */
    BAP_ENOCONV = 4,    /* fit finished; some Newton points hit max_iter (result still valid) */
    BAP_ENOTREADY = 5,  /* bap_poll: the request is not finished yet */
    BAP_EBUSY = 6,      /* bap_submit: admission refused (memory budget or slots full) */
    BAP_ETIMEOUT = 7,   /* a bounded device wait gave up */
    BAP_ESTATE = 8,     /* call out of order, e.g. bap_price before a fit */
    BAP_ECANCELED = 9   /* served request cancelled by bap_cancel */
} bap_status;

/* Payoff Phi(S) at an exercise date (Section 2.2 defines the max-call). */
typedef enum {
    BAP_MAX_CALL = 0,   /* (max_i S_i - K)^+ */
    BAP_BASKET_PUT = 1, /* (K - sum_i w_i S_i)^+ ; with d = 1 the vanilla put */
    BAP_GEO_CALL = 2    /* (prod_i S_i^{w_i} - K)^+ */
} bap_payoff;

typedef enum { BAP_METHOD_IZ = 0, BAP_METHOD_CMC = 1 } bap_method;

#define BAP_MAX_D 10           /* largest number of assets */
#define BAP_MAX_DATES 64       /* largest number of exercise dates */
#define BAP_MAX_STUMPS 256     /* largest number of boosted stumps per date */

/* Market model (Section 2.2 and 3.2): d assets following correlated geometric Brownian motion
 * under the risk-neutral measure, dS_i/S_i = (r - delta_i) dt + sigma_i dW_i, corr(dW) = rho. */
typedef struct bap_model {
    int d;                    /* 1..BAP_MAX_D */
    const double *S0;         /* d spot prices, > 0 */
    const double *sigma;      /* d volatilities, > 0 */
    const double *delta;      /* d dividend yields */
    const double *rho;        /* d*d row-major correlation: symmetric, unit diagonal, positive
                                 definite (checked by an FP64 Cholesky factorisation) */
    double r;                 /* constant interest rate */
    double K;                 /* strike, > 0 */
    double T;                 /* maturity, > 0 */
    int n_dates;              /* N_T exercise dates, 1..BAP_MAX_DATES */
    const double *dates;      /* NULL: t_k = k T / n_dates; else n_dates increasing values in
                                 (0, T] with dates[n_dates-1] == T */
    int payoff;               /* bap_payoff */
    const double *weights;    /* NULL: 1/d each; else d basket weights (basket put, geo call) */
} bap_model;

/* Ibanez-Zapatero parameters (Section 2.2-2.3, Algorithm 1). */
typedef struct bap_iz_params {
    int J;                    /* boundary points per boundary and date (Korobov lattice in the
                                 d-1 other assets; d = 1: J replicate points), 1..8192 */
    int64_t N1;               /* inner paths per continuation estimate, >= 1 */
    double f_tol;             /* stop when |Phi(x) - C(x)| < f_tol (e.g. 1e-6) */
    double x_tol;             /* or when the step or bracket is <= x_tol * max(1, |x|) (e.g. 1e-5) */
    int max_iter;             /* Newton iterations per point, 1..200 (e.g. 50) */
    int degree;               /* boundary polynomial degree 0..3 in the d-1 other assets
                                 (Section 2.1: linear, quadratic or cubic; 3 needs d <= 6;
                                 d = 1 uses 0) */
    uint64_t seed;
    int fixed_point;          /* 1: the paper's literal iteration x <- Phi^-1(C(x)) with |dx| <
                                 fp_eps (Section 2.4); 0: safeguarded Newton */
    double fp_eps;
    int warm_start;           /* 1: each boundary point starts at the later date's fitted boundary
                                 value K B_{m+1}(S_{-p}/K) when that lies inside its initial
                                 bracket (a starting point for Newton, which the paper leaves
                                 open);
                                 0: at the edge of the bracket (max(K, max S_{-p}) for the
                                 max-call); same results to the convergence tolerances */
} bap_iz_params;

/* Picazo CMC parameters (Section 3.2-3.3, Algorithm 2). */
typedef struct bap_cmc_params {
    int J;                    /* training points per date, 2..8192 */
    int64_t N2;               /* inner paths per training point, >= 1 */
    int n_stumps;             /* boosting rounds per date, 1..BAP_MAX_STUMPS */
    uint64_t seed;
    int sampler;              /* training points: 0 independent draws from the law of S_{t_m}
                                 per date; 1 one set of J points walked back from the last
                                 fitted date by a Brownian bridge (Section 3.3), each date's
                                 bridge normals being those the independent draw would use */
    int boost;                /* classifier (Section 3.2 allows either): 0 discrete
                                 AdaBoost on stumps; 1 LogitBoost with regression stumps (then
                                 n_stumps counts rounds, 1..BAP_MAX_STUMPS/2, each stored as a
                                 threshold stump and a constant; J <= 4096; runs on a cluster of
                                 d+1 blocks, EINVAL if the device cannot place it) */
} bap_cmc_params;

typedef struct bap_result {
    double price;             /* Monte Carlo mean of the discounted payoff at tau */
    double se;                /* standard error sqrt(var / n_paths) */
    double var;               /* unbiased sample variance of the discounted payoff */
    double ci95;              /* 1.96 * se */
    int64_t n_paths;
    int64_t path_steps;       /* pricing path-steps actually simulated */
    double fp64_delta;        /* price(FP32 paths) - price(FP64 paths), same counters and rules */
    int n_noconv;             /* boundary points that hit max_iter in the last fit */
    int n_noroot;             /* boundary points without a sign change (left out of the fit) */
    int64_t fit_path_steps;   /* inner path-steps of the last fit */
    double fit_ms;            /* device time of the last fit (CUDA events) */
    double price_ms;          /* device time of the pricing launch */
    int64_t kernel_launches;  /* kernels the library launched for the last fit and this pricing */
    int64_t path_launches;    /* of which path-kernel launches */
    double path_kernel_ms;    /* summed CUDA-event time of those path-kernel launches (only with
                                 bap_set_profiling on; else 0); the FP64 check of
                                 bap_price is not timed */
    double queue_ms;          /* served requests: submit -> admission (host clock) */
    double latency_ms;        /* served requests: submit -> completion (host clock) */
    double phase_ms[4];       /* device time per phase of the paper's time distributions (CUDA
                                 events; the fit's phases only with bap_set_profiling on and a
                                 non-graph launch form, else 0): I&Z [0] [glp] lattice and point
                                 set-up, [1] [calc] Newton passes, [2] [reg] least squares;
                                 CMC [0] 0, [1] [calc] training points and labels, [2] [class]
                                 boosting; both [3] [mc] pricing (= price_ms) */
} bap_result;

typedef struct bap_server_stats {
    int64_t submitted, completed, failed;
    int64_t queued;           /* waiting for admission now */
    int64_t bytes_in_use;     /* estimated device memory of the requests in flight now */
    int64_t peak_bytes, peak_inflight;
    double start_ms;          /* server-thread host time spent starting requests, of which: */
    double load_ms;           /*   giving an option slot its model */
    double fit_enqueue_ms;    /*   enqueueing fits (for I&Z including building the graph) */
    double price_enqueue_ms;  /*   enqueueing pricing */
    double finish_ms;         /* server-thread host time spent finishing requests */
    int64_t cancelled;        /* requests ended by bap_cancel (also counted in failed) */
} bap_server_stats;

typedef struct bap_option bap_option;
typedef struct bap_server bap_server;

/* Create an option: copies and validates the model (an FP64 Cholesky factorisation of rho on
 * the host checks that it is positive definite) and uploads it with the per-date stepping
 * constants.  *out is set on success.  Errors: EINVAL (bad model), ENOMEM, ECUDA. */
bap_status bap_create(const bap_model *model, bap_option **out);

/* Run the option's work on `cuda_stream` (a cudaStream_t; NULL = the legacy default stream). */
bap_status bap_set_stream(bap_option *opt, void *cuda_stream);

/* 1: time every path-kernel launch with a CUDA event pair on the option's stream (reported in
 * bap_result.path_kernel_ms); 0 (default): no per-launch events. */
bap_status bap_set_profiling(bap_option *opt, int on);

/* How bap_fit_boundary issues its work.  1 (default): the whole fit is one CUDA graph, built on
 * the first fit of a parameter set and replayed; each date's Newton loop is a conditional while
 * node whose body runs one Newton pass and then a one-thread kernel that continues the loop only
 * while points remain unconverged (at most max_iter passes), so the loop costs no host round
 * trip and no empty launches.  0: plain form, one launch per Newton pass up to max_iter per date
 * (the graph form falls back to it while profiling is on, and when the graph cannot be built).
 * 2: one cooperative launch per date runs all its Newton passes, a grid-wide barrier between
 * passes; the barrier's wait is bounded, and a barrier that times out makes the fit return
 * ECUDA.  All three forms give bitwise the same fit.  Errors: EINVAL (mode outside 0..2). */
bap_status bap_set_launch_mode(bap_option *opt, int mode);

/* Upper bound, in ns, of one wait at a grid barrier of the cooperative Newton launch (launch
 * form 2).  A block that waits longer gives up, the launch ends, and the fit returns ECUDA with
 * the reason; the option and the device stay usable.  0 (default): 5 s plus 1 ns per inner
 * path-step of the date, far above any real pass.  Small values serve to test that path.
 * Errors: EINVAL (null option). */
bap_status bap_set_wait_limit(bap_option *opt, uint64_t ns);

/* Bounds checks of the checked build (the library compiled with -DBAP_CHECKS, a debug aid in
 * place of a sanitizer): the path kernel checks its item, list, slot, rule-row and trace
 * indices, skips an access that fails and counts it.  *count = failures since the option got its
 * model, *first_code = the first failure's check (1 item, 2 list position, 3 trace index,
 * 4 unit slot, 5 rule row; 0 none).  Always 0 in the normal build.  Waits for the option's
 * stream.  Errors: EINVAL (null argument), ECUDA. */
bap_status bap_debug_checks(bap_option *opt, uint64_t *count, int *first_code);

/* 1 in the checked build, 0 in the normal one. */
int bap_checked_build(void);

/* The launch configuration the library picks for a fit's path launches: for quadratic (or
 * lower) I&Z fits the autotuner's table entry (measured on the target GPU by autotune.py and
 * compiled into the library) nearest to (d, n_items points, N inner paths); otherwise a fixed
 * formula.  It depends on the fit's shape only, so a fit's result is the same alone and served.
 * *unit_paths = paths per warp unit, *paths_per_lane = path slots per lane, *from_table (may be
 * NULL) = 1 if a table entry decided.  Errors: EINVAL. */
bap_status bap_tuned_launch(int d, int method, int degree, int64_t n_items, int64_t N,
                            int *unit_paths, int *paths_per_lane, int *from_table);

/* Cooperative Newton launches of the option use at most 1/share of the device (1, the default,
 * the whole device; the serving loop sets min(max_inflight, 8) so that requests overlap).  The
 * share changes how many blocks run, never the results.  Errors: EINVAL (share outside 1..64). */
bap_status bap_set_grid_share(bap_option *opt, int share);

/* Paths per warp unit of the fits' path launches (I&Z Newton passes, CMC labels): 0 (default)
 * takes the autotuner's choice for the launch shape (bap_tuned_launch); else a multiple of 32 up
 * to 65536.  Longer units spread a unit's fixed set-up and reduction over more paths; shorter ones
 * balance passes with few points.  The choice changes how FP32 partial sums are grouped, so
 * results differ between settings by rounding only.  Errors: EINVAL. */
bap_status bap_set_unit_paths(bap_option *opt, int paths);

/* Path slots per lane of the FP32 kernels with a quadratic (or lower) I&Z boundary: 0 (default)
 * takes the autotuner's choice for the fit's Newton launches (1 elsewhere); 1 or 2 forces it.
 * With 2, every lane advances two paths per step, interleaved, which gives the warp schedulers
 * more independent work; the kernel runs fewer resident blocks.  The choice changes how FP32
 * partial sums are grouped, so results differ between settings by rounding only.
 * Errors: EINVAL (null option, ppl outside 0..2). */
bap_status bap_set_paths_per_lane(bap_option *opt, int ppl);

/* How bap_fit_classifier runs the AdaBoost of each date ([class], Section 3.2; the paper's
 * sequential bottleneck).  3 (default): form 2 for J <= 2048, form 1 above.  2: one 512-thread
 * block with one warp per feature, the sorted orders and weights held in shared memory; used when
 * they fit (J <= 4096 for d = 10), else form 1.  1: a thread-block cluster of d+1 blocks, one per
 * feature, exchanging per-round minima through distributed shared memory; used when the device
 * can place such a cluster, else form 0.  0: one 1024-thread block for all features.  All forms
 * pick the stumps by the same rule on exact fixed-point errors and update the weights by the
 * closed form of the normalised update, so they give identical stumps bit for bit.  LogitBoost
 * (bap_cmc_params.boost = 1) always runs on the cluster.
 * Errors: EINVAL (null option, form outside 0..3). */
bap_status bap_set_boost_form(bap_option *opt, int form);

/* The form the last bap_fit_classifier ran (*form = 2 warp per feature, 1 cluster, 0 one block).
 * Errors: EINVAL (null argument). */
bap_status bap_last_boost_form(const bap_option *opt, int *form);

/* Ibanez-Zapatero fit (Algorithm 1 without [mc]): for m = N_T-1..1, boundary points by
 * device Newton on N1-path continuation estimates, then an FP64 least-squares boundary per
 * (date, boundary).  The fitted rule stays on the device.  Returns OK or ENOCONV. */
bap_status bap_fit_boundary(bap_option *opt, const bap_iz_params *params);

/* CMC fit (Algorithm 2 without [mc]): for m = N_T-1..1, J training points from the law of
 * S_{t_m}, labels from N2-path continuation estimates, AdaBoost stumps on the device. */
bap_status bap_fit_classifier(bap_option *opt, const bap_cmc_params *params);

/* Final pricing ([mc]): n_paths outer paths from S0 under the fitted rule (or, before any fit,
 * exercise at maturity only).  Also reports fp64_delta.  n_paths in 2..2^40. */
bap_status bap_price(bap_option *opt, int64_t n_paths, uint64_t seed, bap_result *out);

/* Rule checkpoint.  Export: with buf == NULL sets *len to the number of doubles needed; else
 * writes min(*len, needed) doubles and sets *len to needed.  Layout (doubles): [kind, n_dates,
 * n_bnd, degree, n_coef, max_stumps, fitted[n_dates+1], then I&Z coef[(n_dates+1)*n_bnd*n_coef]
 * or CMC per date (n_dates+1) x max_stumps x (feat, thr, pol, alpha) plus n_stumps[n_dates+1]].
 * Import accepts the same layout (kind 0 = exercise at maturity only) and returns EINVAL for a
 * shape that does not match the option, a boundary coefficient that is not finite, a stump
 * whose feature is outside 0..d, whose polarity is
 * not +-1 (with a nonzero weight), whose threshold is NaN or whose weight is not finite, or a
 * stump count above max_stumps. */
bap_status bap_export_rules(const bap_option *opt, double *buf, size_t *len);
bap_status bap_import_rules(bap_option *opt, const double *buf, size_t len);

/* Per boundary point (I&Z) or training point (CMC) diagnostics of date m from the last fit:
 * n_items rows of x (I&Z: the boundary point along the pivot; CMC: Phi - C), iterations and
 * status (0 ok, 1 no convergence, 2 no root).  *n_items in: capacity, out: count. */
bap_status bap_fit_points(const bap_option *opt, int m, int *n_items, double *x, int *iters,
                          int *status);

/* Continuation sums for caller-given start points under the option's current rule (debug and
 * parity hook).  For each item i: paths n = 0..N-1 from S_{t_m} = starts[i*d..] with counter
 * item item_ids[i] under stream `purpose` (1 I&Z, 2 CMC).  sums[3i..3i+2] = sum of discounted
 * payoffs, sum of squares, sum of pathwise derivatives w.r.t. starts[i*d + pivots[i]] (pivots
 * may be NULL); steps[i] = path-steps.  1 <= m < n_dates. */
bap_status bap_debug_continuation(bap_option *opt, int m, int purpose, uint64_t seed,
                                  int n_items, const int *item_ids, const int *pivots,
                                  const double *starts, int64_t N, double *sums, int64_t *steps);

/* The same sums with the paths stepped in FP64 (the kernel of bap_price's FP64 re-run): the
 * FP32 path's error of a continuation estimate is the difference of the two on the same
 * counters and rules.  Arguments and errors as bap_debug_continuation. */
bap_status bap_debug_continuation_fp64(bap_option *opt, int m, int purpose, uint64_t seed,
                                       int n_items, const int *item_ids, const int *pivots,
                                       const double *starts, int64_t N, double *sums,
                                       int64_t *steps);

/* Per-path exercise date (n_dates+1 = never) and discounted payoff of one item (parity hook). */
bap_status bap_debug_paths(bap_option *opt, int m, int purpose, uint64_t seed, int item_id,
                           const double *start, int64_t N, int *tau, double *disc_phi);

/* One date of the I&Z fit's Newton loop ([calc], Section 2.3) for caller-given boundary points,
 * under the option's current rules for the later dates (parity hook: with rules imported by
 * bap_import_rules, the points can be compared with another implementation's on the same
 * rules).  Item i starts from starts[i*d..] (the pivot coordinate pivots[i] in 0..d-1 is
 * replaced by the initial iterate, chosen as in the fit; the others must be positive) and uses
 * Philox counter word item_ids[i]; warm_start reads the option's boundary of date m+1.  The
 * launch form is the option's (cooperative, else one launch per pass) with the fit's work split
 * for n_items items and params->N1 paths.  Outputs per item: the final point x, the number of
 * continuation evaluations, the status (0 ok, 1 no convergence, 2 no root) and, if lo and hi
 * are not NULL, the final bracket of the safeguarded Newton iteration (an end not yet found is
 * 0 or +infinity); *path_steps (may be NULL) = inner path-steps taken.  The option's fit scratch
 * is reused (its fit diagnostics and rules are kept).  Errors: EINVAL, ESTATE (the option holds
 * a CMC rule), ECUDA. */
bap_status bap_debug_newton(bap_option *opt, const bap_iz_params *params, int m, int n_items,
                            const int *item_ids, const int *pivots, const double *starts,
                            double *x, int *iters, int *status, double *lo, double *hi,
                            int64_t *path_steps);

/* The I&Z least-squares boundary fit ([reg], Section 2.2) of one date on caller-given points
 * (parity hook).  n_bnd = d for the max-call with d > 1, else 1; boundary b holds points
 * b*J .. b*J+J-1: starts[(b*J+j)*d..] (the other assets' values; the pivot's entry is ignored),
 * x[b*J+j] the point along the pivot and status[b*J+j] (2 = no root: left out).  coef receives
 * n_bnd x n_basis(d-1, degree) FP64 coefficients of x/K in the monomials of y/K, in the order
 * [1, y_a, y_a y_b (a <= b), y_a y_b y_c (a <= b <= c)], exactly as bap_export_rules stores a
 * date.  The option's rules are not touched.  Errors: EINVAL, ECUDA. */
bap_status bap_debug_ls_fit(bap_option *opt, int degree, int J, const double *starts,
                            const double *x, const int *status, double *coef);

/* The CMC boosting of one date ([class], Section 3.2) on caller-given training points X (J x d,
 * positive) and labels (+1 exercise / -1 continue), in the option's boosting form (parity hook).
 * The stumps become the option's rule of date m (if the option does not hold a CMC rule with
 * room for params->n_stumps stumps, or twice that for LogitBoost, an empty one is set up
 * first).  *n_stumps = stumps fitted; stumps receives max_stumps x (feature, threshold,
 * polarity, alpha), the layout of bap_export_rules.  Errors: EINVAL, ECUDA. */
bap_status bap_debug_boost(bap_option *opt, const bap_cmc_params *params, int m, const double *X,
                           const int *labels, int *n_stumps, double *stumps);

/* Continuation sums that allocate no device memory.  The paper has no counterpart to this call.
 * It is for callers that cannot allocate device memory while they run -- code inside a host
 * framework whose allocator owns all of the GPU's memory, or a latency-bound loop that must not
 * call cudaMalloc or cudaFree (both can block on the whole device) -- and that bring their own
 * device buffers.  It computes what bap_debug_continuation computes, but:
 *   - every array is a DEVICE pointer: d_item_ids and d_pivots (n_items ints; d_pivots may be
 *     NULL), d_starts (n_items*d doubles), d_sums (n_items*3 doubles), d_steps (n_items);
 *   - a pivot must lie in -1..d-1 and every start coordinate must be positive.  The inputs are
 *     checked on the device: an item that breaks either rule gets NaN sums and steps = -1 (its
 *     pivot is treated as -1, so no access leaves the caller's buffers); the other items are
 *     unaffected.  The call itself cannot see the device data and returns OK;
 *   - the call only enqueues work on the option's stream and returns.  The inputs must be
 *     complete with respect to that stream when the call is made: if they were written on
 *     another stream, synchronize it or make the option's stream wait on an event first.
 *     Synchronize the option's stream before reading d_sums and d_steps;
 *   - its scratch is a fixed 4 MiB array in the library's device image (one per GPU that loads
 *     the library, held until the process exits).  A call needs about 32 bytes per
 *     (item, unit of up to 2048 paths) plus 4 bytes per item; larger calls return BAP_EINVAL;
 *   - every call looks up the array's address on the current device (which must be the
 *     option's, as for every call on the option); the first lookup on a device may load the
 *     library's device image there, so make the first call before any stream capture;
 *   - all calls share the array, and it keeps the last call's contents (the call clears what it
 *     needs zeroed): calls whose work overlaps on the GPU -- on different streams, or different
 *     options on one device -- race on it and corrupt each other's sums.  Serialize them. */
bap_status bap_continuation_static(bap_option *opt, int m, int purpose, uint64_t seed,
                                   int n_items, const int *d_item_ids, const int *d_pivots,
                                   const double *d_starts, int64_t N, double *d_sums,
                                   int64_t *d_steps);

/* Raw Philox4x32-10 words and the Box-Muller normals of the counters (n, w1, 4*step + c),
 * n = 0..count-1, under key (seed, purpose, m) (parity hook; no option needed).  words:
 * count * 4 * ceil(d/4) uint32 (may be NULL); z: count * d doubles converted from the FP32
 * normals (may be NULL). */
bap_status bap_debug_rng(uint64_t seed, int purpose, int m, uint32_t w1, uint32_t step, int d,
                         int64_t count, uint32_t *words, double *z);

/* ---- Serving (continuous batching) ----------------------------------------------------------
 * A server owns a thread that admits submitted requests while the requests in flight number at
 * most max_inflight and their estimated device memory stays within device_mem_budget bytes.  It
 * runs each admitted request -- create, fit (I&Z graph or CMC), price -- on a stream of its own,
 * so requests overlap on the device; when one finishes its slot and memory go to the next in
 * the queue.  A request's result depends only on its inputs: it is the same, bitwise, as the
 * same calls made alone through bap_create / bap_fit_* / bap_price.  All server calls are
 * thread safe.  The server uses the device current at bap_server_create. */

/* Errors: EINVAL (budget < 1 MiB, max_inflight outside 1..1024), ECUDA (no device), ENOMEM.
 * Each request in flight runs on its own stream: set CUDA_DEVICE_MAX_CONNECTIONS=32 in the
 * environment before the process creates its CUDA context, else CUDA multiplexes the streams
 * onto 8 hardware queues and requests wait for each other (the Python binding sets it at
 * import unless it is already set). */
bap_status bap_server_create(size_t device_mem_budget, int max_inflight, bap_server **out);

/* Launch form of the I&Z fits the server runs (see bap_set_launch_mode).  Default 2 (one
 * cooperative launch per date, on at most 1/min(max_inflight, 8) of the device): each request
 * builds its fit once, so a graph's build and release cost more host time than its launches
 * save, and the plain form's max_iter launches per date fill the stream's launch queue. */
bap_status bap_server_set_launch_mode(bap_server *srv, int mode);

/* Queue a request: method BAP_METHOD_IZ with params -> bap_iz_params, or BAP_METHOD_CMC with
 * params -> bap_cmc_params; then pricing with n_paths paths and `seed`.  The model and params
 * are copied.  *ticket identifies the request.  Errors: EINVAL (bad arguments, checked as
 * bap_create / bap_fit_* would), EBUSY (the request alone needs more than the budget). */
bap_status bap_submit(bap_server *srv, const bap_model *model, int method, const void *params,
                      int64_t n_paths, uint64_t seed, uint64_t *ticket);

/* Non-blocking: BAP_ENOTREADY while queued or running; otherwise the request's final status
 * (OK, ENOCONV, or its error) with *out filled (may be NULL), after which the ticket is gone.
 * EINVAL for an unknown ticket. */
bap_status bap_poll(bap_server *srv, uint64_t ticket, bap_result *out);

/* Cancel a request that has not been collected.  Queued: it is dropped at once.  Running: the
 * server sets the request's device abort flag (the one the cooperative Newton launch checks at
 * every grid barrier, so an I&Z fit in launch form 2 stops at its next pass) and discards the
 * result when the request's work ends.  Either way bap_poll / bap_wait then return ECANCELED.
 * A request already finished keeps its result (returns ESTATE).  Thread safe.
 * Errors: EINVAL (null server, unknown ticket), ESTATE (already finished). */
bap_status bap_cancel(bap_server *srv, uint64_t ticket);

/* As bap_poll, but waits up to timeout_s seconds; BAP_ETIMEOUT if still not done. */
bap_status bap_wait(bap_server *srv, uint64_t ticket, double timeout_s, bap_result *out);

bap_status bap_server_get_stats(bap_server *srv, bap_server_stats *out);

/* Finishes every queued and running request, then stops the thread and frees everything
 * (results not collected are discarded). NULL is ignored. */
void bap_server_destroy(bap_server *srv);

/* Release an option and its device memory (NULL is ignored). */
void bap_destroy(bap_option *opt);

/* Message of the last failed call on this thread ("" if none). */
const char *bap_last_error(void);

/* Library version string. */
const char *bap_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BAP_H */
