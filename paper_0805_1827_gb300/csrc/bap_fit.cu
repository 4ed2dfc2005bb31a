// bap_fit.cu -- device kernels around the path kernel: model set-up, the Korobov lattice
// ([glp]), boundary-point set-up, the FP64 least-squares boundary fit ([reg]), CMC training
// points and device AdaBoost ([class]), and the staging of fitted rules for the path kernel.
#include "bap_fit.cuh"

#include <cfloat>

#include <cooperative_groups.h>

namespace bap {

// ---------------------------------------------------------------------------------------------
// [glp] Korobov rank-1 lattice (Section 2.3): the multiplier a minimising the P_2 figure of
// merit -1 + (1/J) sum_j prod_k (1 + 2 pi^2 B_2({j a^k / J})), B_2(x) = x^2 - x + 1/6, over
// a in [1, J) coprime to J; ties within 1e-9 (relative) go to the smallest a.

__device__ inline unsigned gcd_u(unsigned a, unsigned b) {
    while (b) { unsigned t = a % b; a = b; b = t; }
    return a;
}

__global__ void korobov_merit_kernel(int J, int s, double* merit) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int a = warp + 1;
    if (a >= J) return;
    if (gcd_u((unsigned)a, (unsigned)J) != 1u) {
        if (lane == 0) merit[a] = INFINITY;
        return;
    }
    unsigned long long g[MAXD];
    g[0] = 1;
    for (int k = 1; k < s; ++k) g[k] = (g[k - 1] * (unsigned long long)a) % (unsigned long long)J;
    const double c2 = 2.0 * 9.869604401089358;   // 2 pi^2
    double sum = 0.0;
    for (int j = lane; j < J; j += 32) {
        double prod = 1.0;
        for (int k = 0; k < s; ++k) {
            const double u = (double)(((unsigned long long)j * g[k]) % (unsigned long long)J) / (double)J;
            prod *= 1.0 + c2 * (u * u - u + 1.0 / 6.0);
        }
        sum += prod;
    }
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off);
    if (lane == 0) merit[a] = -1.0 + sum / (double)J;
}

__global__ void korobov_pick_kernel(int J, int s, const double* merit, int* out_a) {
    __shared__ double smin[32];
    __shared__ int sidx[32];
    if (s <= 1 || J <= 2) {
        if (threadIdx.x == 0) *out_a = 1;
        return;
    }
    double mn = INFINITY;
    for (int a = 1 + threadIdx.x; a < J; a += blockDim.x) mn = fmin(mn, merit[a]);
    for (int off = 16; off > 0; off >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, off));
    if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = mn;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < blockDim.x / 32 ? smin[threadIdx.x] : INFINITY;
        for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, off));
        if (threadIdx.x == 0) smin[0] = v;
    }
    __syncthreads();
    const double vmin = smin[0];
    const double tol = 1e-9 * fmax(fabs(vmin), 1e-300);
    int best = J;
    for (int a = 1 + threadIdx.x; a < J; a += blockDim.x)
        if (merit[a] <= vmin + tol && a < best) best = a;
    for (int off = 16; off > 0; off >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, off));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sidx[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        int b = J;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) b = min(b, sidx[w]);
        *out_a = b < J ? b : 1;
    }
}

// ---------------------------------------------------------------------------------------------
// I&Z items of date m (item = b*J + j): the other assets at the lognormal quantiles of the
// shifted lattice point frac(j g / J + 1/(2J)), the pivot at the Newton start, and the bracket.

// Newton state of one boundary point whose other coordinates S[q], q != p, are set: the initial
// bracket and iterate (Section 2.3: Newton's iterations from an approximate point), warm-started
// at the later date's fitted boundary when asked; writes the initial iterate to S[p] and returns
// whether the point needs evaluations (false: no root, e.g. a put whose other assets alone
// exceed the strike).  b = the boundary whose later-date coefficients seed a warm start.
__device__ bool newton_item_init(const DevModel* M, int m, int n_bnd, int b, int p, double* S,
                                 ItemState& st, const double* coef64, int n_coef, int degree,
                                 const int* fitted, int warm_start) {
    const int d = M->d, s = d - 1;
    const double K = M->K;
    st.iters = 0;
    st.status = ST_OK;
    st.done = 0;
    st.pivot = p;
    st.dx_old = INFINITY;
    st.dx = INFINITY;
    bool live = true;
    if (M->payoff == BAP_MAX_CALL) {
        double mx = K;
        for (int q = 0; q < d; ++q)
            if (q != p && S[q] > mx) mx = S[q];
        st.lo = mx;
        st.hi = INFINITY;
        st.x = mx * (1.0 + 1e-3);
    } else if (M->payoff == BAP_GEO_CALL) {
        double lg = log(K);
        for (int q = 0; q < d; ++q)
            if (q != p) lg -= M->w[q] * log(S[q]);
        st.lo = exp(lg / M->w[p]);
        st.hi = INFINITY;
        st.x = st.lo * (1.0 + 1e-3);
    } else {
        double top = K;
        for (int q = 0; q < d; ++q)
            if (q != p) top -= M->w[q] * S[q];
        top /= M->w[p];
        if (!(top > 0)) {
            st.x = 0.0;
            st.lo = 0.0;
            st.hi = 0.0;
            st.status = ST_NOROOT;
            st.done = 1;
            live = false;
        } else {
            st.lo = 0.0;
            st.hi = top;
            st.x = top * (1.0 - 1e-3);
        }
    }
    // warm start: the later date's fitted boundary K B_{m+1}(S_{-p}/K) (FP64, basis order
    // [1, y_a, y_a y_b, y_a y_b y_c]) when it lies inside the initial bracket
    if (live && warm_start && m + 1 < M->n_dates && fitted[m + 1]) {
        double y[MAXD];
        int t = 0;
        for (int q = 0; q < d; ++q)
            if (q != p) y[t++] = S[q] / K;
        const double* c = coef64 + ((size_t)(m + 1) * n_bnd + b) * n_coef;
        double B = 0.0;
        int i = 0;
        B += c[i++] * 1.0;
        if (degree >= 1)
            for (int a = 0; a < s; ++a) B += c[i++] * y[a];
        if (degree >= 2)
            for (int a = 0; a < s; ++a)
                for (int e = a; e < s; ++e) B += c[i++] * (y[a] * y[e]);
        if (degree >= 3)
            for (int a = 0; a < s; ++a)
                for (int e = a; e < s; ++e)
                    for (int g3 = e; g3 < s; ++g3) B += c[i++] * (y[a] * y[e] * y[g3]);
        const double xw = K * B;
        if (xw > st.lo && xw < st.hi) st.x = xw;
    }
    S[p] = st.x;
    return live;
}

// (float) log2 of an item's start point, the form the FP32 path kernels read (l0f).
__device__ inline void store_log_start(const double* S, int d, float* l0f) {
    for (int q = 0; q < d; ++q) l0f[q] = (float)log2(S[q]);
}

__global__ void iz_setup_kernel(const DevModel* M, int m, int J, int n_bnd, const int* korobov_a,
                                double* start, ItemState* state, int* pivot, int* active,
                                int* count, const double* coef64, int n_coef, int degree,
                                const int* fitted, int warm_start, float* l0f) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= n_bnd * J) return;
    const int d = M->d;
    const int b = item / J, j = item - b * J;
    const int p = n_bnd > 1 ? b : 0;
    const double tm = M->t[m];
    double* S = start + (size_t)item * d;
    unsigned long long g = 1;
    const unsigned long long a = (unsigned long long)(*korobov_a);
    for (int q = 0; q < d; ++q) {
        if (q == p) continue;
        const double u = ((double)(((unsigned long long)j * g) % (unsigned long long)J) + 0.5) / (double)J;
        const double mu = M->r - M->delta[q] - 0.5 * M->sigma[q] * M->sigma[q];
        S[q] = M->S0[q] * exp(mu * tm + M->sigma[q] * sqrt(tm) * normcdfinv(u));
        g = (g * a) % (unsigned long long)J;
    }
    ItemState st;
    const bool live = newton_item_init(M, m, n_bnd, b, p, S, st, coef64, n_coef, degree, fitted,
                                       warm_start);
    state[item] = st;
    pivot[item] = p;
    store_log_start(S, d, l0f + (size_t)item * d);
    if (live) {
        const int pos = atomicAdd(count, 1);
        active[pos] = item;
    }
}

// The same set-up for caller-given points (the parity hook bap_debug_newton): item i starts from
// starts_in[i] (its pivot coordinate is replaced by the initial iterate), with pivot pivots_in[i]
// and counter word ctr_in[i].  Items enter the first pass's list in index order, so the pass's
// work split does not depend on thread scheduling.
__global__ void newton_items_setup_kernel(const DevModel* M, int m, int n_items, int n_bnd,
                                          const double* starts_in, const int* pivots_in,
                                          const int* ctr_in, double* start, ItemState* state,
                                          int* pivot, int* ctr_item, int* live_flag,
                                          const double* coef64, int n_coef, int degree,
                                          const int* fitted, int warm_start, float* l0f) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= n_items) return;
    const int d = M->d;
    const int p = pivots_in[item];
    double* S = start + (size_t)item * d;
    for (int q = 0; q < d; ++q) S[q] = starts_in[(size_t)item * d + q];
    ItemState st;
    const bool live = newton_item_init(M, m, n_bnd, n_bnd > 1 ? p : 0, p, S, st, coef64, n_coef,
                                       degree, fitted, warm_start);
    state[item] = st;
    pivot[item] = p;
    ctr_item[item] = ctr_in[item];
    live_flag[item] = live ? 1 : 0;
    store_log_start(S, d, l0f + (size_t)item * d);
}

// Compacts the live items into the first pass's list in index order (one block).
__global__ void newton_items_list_kernel(const int* live_flag, int n_items, int* active, int* count) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int c = 0;
    for (int i = 0; i < n_items; ++i)
        if (live_flag[i]) active[c++] = i;
    *count = c;
}

// ---------------------------------------------------------------------------------------------
// Staging of an I&Z boundary (date m, boundary b) for the path kernel: coefficients of
// x/K = B(y/K) in [1, y_a, y_a y_b (a<=b)] order (for the given degree) become the full
// quadratic Horner layout [K c_0, for a: c_a, c_ab / K (b = a..s-1)] of B''(S) = K B(S/K) in
// price units, zero-filled for lower degrees and padded to iz_stage_stride(s + 1) values.

__device__ void stage_iz_one(const double* c, int s, int degree, double K, int p, float* out_f,
                             double* out_d) {
    // x = K B(y/K) with B = sum of c_i times the monomials of y/K: in price units the constant
    // is K c_0, the linear terms keep c_t, the quadratic c_tu / K, the cubic c_tuv / K^2.
    const int stride = iz_stride(s + 1, degree);
    for (int i = 0; i < stride; ++i) { out_f[i] = 0.f; out_d[i] = 0.0; }
    out_f[0] = (float)(K * c[0]);
    out_d[0] = K * c[0];
    // positions of the quadratic and cubic coefficients in the basis order [1, y_a, y_a y_b
    // (a <= b), y_a y_b y_c (a <= b <= c)]
    const int q0 = 1 + s, c0 = 1 + s + s * (s + 1) / 2;
    auto qpos = [&](int t, int u) {        // index of y_t y_u, t <= u
        int k = 0;
        for (int a = 0; a < t; ++a) k += s - a;
        return q0 + k + (u - t);
    };
    if (degree <= 2) {
        // Up to quadratic: the polynomial in all d = s + 1 prices, with zero terms for the pivot
        // asset p, nested for Horner: c_0, then for each asset t: c_t and, for each u >= t, c_tu:
        //   B = c_0 + sum_t S_t (c_t + sum_{u>=t} c_tu S_u).
        // The path kernel then evaluates it on the prices as they are, with no reordering.
        const int d = s + 1;
        int o = 1;
        for (int t = 0; t < d; ++t) {
            const int yt = t < p ? t : t - 1;
            const double lin = (degree >= 1 && t != p) ? c[1 + yt] : 0.0;
            out_f[o] = (float)lin;
            out_d[o] = lin;
            ++o;
            for (int u = t; u < d; ++u, ++o) {
                const int yu = u < p ? u : u - 1;
                const double q = (degree >= 2 && t != p && u != p) ? c[qpos(yt, yu)] / K : 0.0;
                out_f[o] = (float)q;
                out_d[o] = q;
            }
        }
        return;
    }
    // Cubic: the polynomial in the d - 1 other prices y (in asset order), nested for Horner:
    // c_0, then for each t: c_t and, for each u >= t, c_tu followed by its c_tuv for v >= u:
    //   B = c_0 + sum_t y_t (c_t + sum_{u>=t} y_u (c_tu + sum_{v>=u} y_v c_tuv)).
    auto cpos = [&](int t, int u, int v) { // index of y_t y_u y_v, t <= u <= v
        int k = 0;
        for (int a = 0; a < s; ++a)
            for (int b = a; b < s; ++b)
                for (int e = b; e < s; ++e) {
                    if (a == t && b == u && e == v) return c0 + k;
                    ++k;
                }
        return c0;
    };
    int o = 1;
    for (int t = 0; t < s; ++t) {
        const double lin = c[1 + t];
        out_f[o] = (float)lin;
        out_d[o] = lin;
        ++o;
        for (int u = t; u < s; ++u) {
            const double q = c[qpos(t, u)] / K;
            out_f[o] = (float)q;
            out_d[o] = q;
            ++o;
            for (int v = u; v < s; ++v, ++o) {
                const double cu = c[cpos(t, u, v)] / (K * K);
                out_f[o] = (float)cu;
                out_d[o] = cu;
            }
        }
    }
}

__global__ void stage_iz_kernel(const double* coef64, int n_dates, int n_bnd, int n_coef, int s,
                                int degree, double K, float* coef_f, double* coef_d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (n_dates + 1) * n_bnd) return;
    const size_t so = (size_t)i * iz_stride(s + 1, degree);
    const int b = i % n_bnd;
    stage_iz_one(coef64 + (size_t)i * n_coef, s, degree, K, n_bnd > 1 ? b : 0, coef_f + so,
                 coef_d + so);
}

// ---------------------------------------------------------------------------------------------
// [reg] Least squares of x/K on the polynomial basis of y/K for boundary b of date m (FP64).
// Points with status "no root" are left out; fewer points than coefficients -> degree 0 (their
// mean); no points -> "never exercise".  Normal equations on the diagonally equilibrated Gram
// matrix, solved by Cholesky and corrected by one refinement step on the residual; a Cholesky
// failure also falls back to the mean.

__device__ inline double basis_val(const double* y, int bi, int bj, int bk) {
    const double a = bi < 0 ? 1.0 : y[bi];
    const double b = bj < 0 ? 1.0 : y[bj];
    if (bk < 0) return a * b;
    return a * b * y[bk];
}

__global__ void __launch_bounds__(kLsThreads) ls_fit_kernel(const DevModel* M, int m, int J, int n_bnd, int degree, int n_coef,
                              const double* start, const ItemState* state, double* coef64,
                              float* coef_f, double* coef_d, int* fitted) {
    const int b = blockIdx.x;
    const int d = M->d, s = d - 1;
    const int p = n_bnd > 1 ? b : 0;
    const double K = M->K;
    __shared__ int bi[MAXCOEF], bj[MAXCOEF], bk[MAXCOEF];
    __shared__ double G[MAXCOEF * MAXCOEF];
    __shared__ double rhs[MAXCOEF];
    __shared__ double red[32];
    __shared__ int red_n[32];
    __shared__ double coef[MAXCOEF];
    const int P = n_coef;
    if (threadIdx.x == 0) {
        int o = 0;
        bi[o] = -1; bj[o] = -1; bk[o] = -1; ++o;
        if (degree >= 1)
            for (int t = 0; t < s; ++t) { bi[o] = t; bj[o] = -1; bk[o] = -1; ++o; }
        if (degree >= 2)
            for (int t = 0; t < s; ++t)
                for (int u = t; u < s; ++u) { bi[o] = t; bj[o] = u; bk[o] = -1; ++o; }
        if (degree >= 3)
            for (int t = 0; t < s; ++t)
                for (int u = t; u < s; ++u)
                    for (int v = u; v < s; ++v) { bi[o] = t; bj[o] = u; bk[o] = v; ++o; }
    }
    __syncthreads();
    // count of used points and their mean
    double sx = 0.0;
    int nu = 0;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        const int item = b * J + j;
        if (state[item].status != ST_NOROOT) {
            sx += state[item].x / K;
            ++nu;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, off);
        nu += __shfl_down_sync(0xffffffffu, nu, off);
    }
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = sx; red_n[threadIdx.x >> 5] = nu; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0; int n = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) { t += red[w]; n += red_n[w]; }
        red[0] = t; red_n[0] = n;
    }
    __syncthreads();
    const int n_used = red_n[0];
    const double mean = n_used > 0 ? red[0] / n_used : 0.0;
    bool use_mean = n_used < P;
    if (!use_mean) {
        // Normal equations: entry (r, c) of G (and r of the right side, column P below) is the
        // sum over the used points, in point order, of basis_r * basis_c.  The basis values of
        // kChunk points at a time are staged in shared memory once; each thread keeps the sums
        // of its own entries e = threadIdx.x + k * blockDim.x.
        const int npair = P * (P + 1) / 2;
        constexpr int kChunk = 32;
        constexpr int kEPT = (MAXCOEF * (MAXCOEF + 1) / 2 + MAXCOEF + kLsThreads - 1) / kLsThreads;
        __shared__ double Bs[kChunk][MAXCOEF + 1];
        __shared__ int Bu[kChunk];
        int er[kEPT], ec[kEPT];
        double acc[kEPT];
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const int e = threadIdx.x + k * kLsThreads;
            int r = -1, c = -1;
            if (e < npair) {
                int rem = e;
                r = 0;
                while (rem >= P - r) { rem -= P - r; ++r; }
                c = r + rem;
            } else if (e < npair + P) {
                r = e - npair;
                c = P;
            }
            er[k] = r;
            ec[k] = c;
            acc[k] = 0.0;
        }
        for (int j0 = 0; j0 < J; j0 += kChunk) {
            for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
                const int j = j0 + t;
                int used = 0;
                if (j < J) {
                    const int item = b * J + j;
                    if (state[item].status != ST_NOROOT) {
                        used = 1;
                        const double* S = start + (size_t)item * d;
                        double y[MAXD];
                        int u = 0;
                        for (int q = 0; q < d; ++q)
                            if (q != p) y[u++] = S[q] / K;
                        for (int r = 0; r < P; ++r) Bs[t][r] = basis_val(y, bi[r], bj[r], bk[r]);
                        Bs[t][P] = state[item].x / K;
                    }
                }
                Bu[t] = used;
            }
            __syncthreads();
            // a thread's entries are a prefix of its slots: stop at the first empty one, so that
            // warps without entries issue no FP64 work (the FP64 pipe is 1/64 of the FP32 rate)
            for (int t = 0; t < kChunk; ++t) {
                if (!Bu[t]) continue;
#pragma unroll
                for (int k = 0; k < kEPT; ++k) {
                    if (er[k] < 0) break;
                    acc[k] += Bs[t][er[k]] * Bs[t][ec[k]];
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const int r = er[k], c = ec[k];
            if (r < 0) continue;
            if (c < P) { G[r * P + c] = acc[k]; G[c * P + r] = acc[k]; }
            else rhs[r] = acc[k];
        }
        __syncthreads();
        // Scale to a unit diagonal, factor G = L L^T (lower, in place) with the rank test on the
        // pivots, and solve.  The block shares the work; every entry receives the same
        // operations in the same order as in a one-thread left-looking factorisation (entry
        // (i, j) starts from its scaled value and subtracts L[i][k] L[j][k] for k = 0, 1, ...,
        // j - 1), so the coefficients are those of that sequential form bit for bit.
        __shared__ double dsc[MAXCOEF];
        __shared__ double s_l;
        __shared__ int s_ok;
        const int tid = threadIdx.x, nth = blockDim.x;
        if (tid == 0) s_ok = 1;
        __syncthreads();
        for (int i = tid; i < P; i += nth) {
            dsc[i] = G[i * P + i] > 0 ? 1.0 / sqrt(G[i * P + i]) : 0.0;
            if (dsc[i] == 0.0) s_ok = 0;
        }
        __syncthreads();
        bool ok = s_ok != 0;
        if (ok) {
            for (int e = tid; e < P * P; e += nth) G[e] *= dsc[e / P] * dsc[e % P];
            __syncthreads();
            // right-looking: column jj's pivot, the column below it, then the trailing triangle
            for (int jj = 0; jj < P; ++jj) {
                if (tid == 0) {
                    const double v = G[jj * P + jj];
                    if (!(v > 1e-13)) {
                        s_ok = 0;
                    } else {
                        s_l = sqrt(v);
                        G[jj * P + jj] = s_l;
                    }
                }
                __syncthreads();
                if (!s_ok) break;
                const double l = s_l;
                for (int i = jj + 1 + tid; i < P; i += nth) G[i * P + jj] = G[i * P + jj] / l;
                __syncthreads();
                const int n = P - 1 - jj;                 // trailing rows and columns jj+1..P-1
                for (int e = tid; e < n * (n + 1) / 2; e += nth) {
                    int i = 0, rem = e;                   // row i (0-based in the trailing part)
                    while (rem > i) { rem -= i + 1; ++i; }
                    const int r = jj + 1 + i, c = jj + 1 + rem;      // c <= r
                    G[r * P + c] -= G[r * P + jj] * G[c * P + jj];
                }
                __syncthreads();
            }
            ok = s_ok != 0;
        }
        if (ok) {
            // forward: z = L^-1 (dsc * rhs), column by column (row i subtracts in k order)
            for (int i = tid; i < P; i += nth) rhs[i] *= dsc[i];
            __syncthreads();
            for (int k = 0; k < P; ++k) {
                if (tid == 0) rhs[k] = rhs[k] / G[k * P + k];
                __syncthreads();
                const double zk = rhs[k];
                for (int i = k + 1 + tid; i < P; i += nth) rhs[i] -= G[i * P + k] * zk;
                __syncthreads();
            }
            // backward: L^T coef = z, one thread (each row sums in ascending k)
            if (tid == 0) {
                for (int i = P - 1; i >= 0; --i) {
                    double v = rhs[i];
                    for (int k = i + 1; k < P; ++k) v -= G[k * P + i] * coef[k];
                    coef[i] = v / G[i * P + i];
                }
                for (int i = 0; i < P; ++i) coef[i] *= dsc[i];
            }
            __syncthreads();
            // One step of refinement with the same factor (corrected semi-normal equations,
            // Bjorck): the residual r = x - A c of the used points in FP64, then A^T r solved as
            // above and added to c.  Normal equations alone leave a forward error of order
            // cond(A)^2 u; the corrected step brings it to order cond(A) u, as a QR
            // factorisation of A would, for cond(A)^2 u < 1.
            double gacc = 0.0;                    // thread i < P: entry i of A^T r, point order
            for (int j0 = 0; j0 < J; j0 += kChunk) {
                for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
                    const int j = j0 + t;
                    int used = 0;
                    if (j < J) {
                        const int item = b * J + j;
                        if (state[item].status != ST_NOROOT) {
                            used = 1;
                            const double* S = start + (size_t)item * d;
                            double y[MAXD];
                            int u = 0;
                            for (int q = 0; q < d; ++q)
                                if (q != p) y[u++] = S[q] / K;
                            double r = state[item].x / K;
                            for (int i = 0; i < P; ++i) {
                                const double bv = basis_val(y, bi[i], bj[i], bk[i]);
                                Bs[t][i] = bv;
                                r -= coef[i] * bv;
                            }
                            Bs[t][P] = r;
                        }
                    }
                    Bu[t] = used;
                }
                __syncthreads();
                if (tid < P)
                    for (int t = 0; t < kChunk; ++t)
                        if (Bu[t]) gacc += Bs[t][tid] * Bs[t][P];
                __syncthreads();
            }
            if (tid < P) rhs[tid] = gacc * dsc[tid];
            __syncthreads();
            for (int k = 0; k < P; ++k) {
                if (tid == 0) rhs[k] = rhs[k] / G[k * P + k];
                __syncthreads();
                const double zk = rhs[k];
                for (int i = k + 1 + tid; i < P; i += nth) rhs[i] -= G[i * P + k] * zk;
                __syncthreads();
            }
            if (tid == 0) {
                double dlt[MAXCOEF];
                for (int i = P - 1; i >= 0; --i) {
                    double v = rhs[i];
                    for (int k = i + 1; k < P; ++k) v -= G[k * P + i] * dlt[k];
                    dlt[i] = v / G[i * P + i];
                }
                for (int i = 0; i < P; ++i) coef[i] += dlt[i] * dsc[i];
            }
        } else if (tid == 0) {
            for (int i = 0; i < P; ++i) coef[i] = 0.0;
            coef[0] = mean;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (n_used == 0) {
            for (int i = 0; i < P; ++i) coef[i] = 0.0;
            coef[0] = M->payoff == BAP_BASKET_PUT ? -1.0 : 1e30;
        } else if (use_mean) {
            for (int i = 0; i < P; ++i) coef[i] = 0.0;
            coef[0] = mean;
        }
        const size_t o = ((size_t)m * n_bnd + b) * P;
        for (int i = 0; i < P; ++i) coef64[o + i] = coef[i];
        const size_t so = ((size_t)m * n_bnd + b) * iz_stride(d, degree);
        stage_iz_one(coef64 + o, s, degree, K, p, coef_f + so, coef_d + so);
        if (b == 0) fitted[m] = 1;
    }
}

// ---------------------------------------------------------------------------------------------
// CMC training points of date m: S = S_0 exp(mu t_m + sqrt(t_m) L z) with FP64 Box-Muller
// normals of counter (j, 0, c, 0) under the TRAIN stream (reading of Section 3.3: independent
// draws from the law of S_{t_m}).

__global__ void train_points_kernel(const DevModel* M, int m, RoundKeys rk, int J, double* start,
                                    int* ctr_item, double* W, int bridge_from_next) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    const int d = M->d;
    double z[MAXD + 3];
    for (int c = 0; c < (d + 3) / 4; ++c) {
        const uint4 x = philox((uint32_t)j, 0u, (uint32_t)c, 0u, rk);
        double a0, a1;
        PathMath<double>::box_muller(x.x, x.y, a0, a1);
        z[4 * c] = a0;
        z[4 * c + 1] = a1;
        PathMath<double>::box_muller(x.z, x.w, a0, a1);
        z[4 * c + 2] = a0;
        z[4 * c + 3] = a1;
    }
    const double tm = M->t[m];
    if (W == nullptr) {
        for (int q = 0; q < d; ++q) {
            double wq = 0.0;
            for (int i = 0; i <= q; ++i) wq += M->L[q * MAXD + i] * z[i];
            const double mu = M->r - M->delta[q] - 0.5 * M->sigma[q] * M->sigma[q];
            start[(size_t)j * d + q] = M->S0[q] * exp(mu * tm + M->sigma[q] * sqrt(tm) * wq);
        }
    } else {
        // Brownian bridge (Section 3.3): W_m = a W_{m+1} + b L z with a = t_m / t_{m+1} and
        // b = sqrt(t_m (t_{m+1} - t_m) / t_{m+1}); at the last fitted date a = 0, b = sqrt(t_m).
        // W holds this point's W_{m+1} on entry and W_m on exit.
        double a = 0.0, b = sqrt(tm);
        if (bridge_from_next) {
            const double tn = M->t[m + 1];
            a = tm / tn;
            b = sqrt(tm * (tn - tm) / tn);
        }
        for (int q = 0; q < d; ++q) {
            double lz = 0.0;
            for (int i = 0; i <= q; ++i) lz += M->L[q * MAXD + i] * z[i];
            const double w = b * lz + (bridge_from_next ? a * W[(size_t)j * d + q] : 0.0);
            const double mu = M->r - M->delta[q] - 0.5 * M->sigma[q] * M->sigma[q];
            W[(size_t)j * d + q] = w;
            start[(size_t)j * d + q] = M->S0[q] * exp(mu * tm + M->sigma[q] * w);
        }
    }
    ctr_item[j] = j;
}

// ---------------------------------------------------------------------------------------------
// CMC rule staging for one date: constant stumps fold into F0; per feature the finite
// thresholds sorted ascending and the step table T_f[c] = sum_{i<c} alpha_i pol_i -
// sum_{i>=c} alpha_i pol_i, so F(S) = F0 + sum_f T_f[#{thresholds < x_f}], kept at the distinct
// thresholds only (the record layout is described with CMC_SLOTS).

// One feature's block of a staged CMC record (in the record's own precision): the distinct
// sorted thresholds (equal in that precision merged) and the step value below each and above
// the last one.  A step value is the sum of the feature's votes at a value just above that many
// distinct thresholds: stump i votes +pol_i above its threshold and -pol_i at or below it, so
// with pre = the alpha-weighted votes of the stumps below, the sum is 2 pre - (all of them).
template <typename Real>
__device__ void stage_cmc_feature(int f, int n, const int* idx, const double* thr,
                                  const int* pol, const double* alpha, double tot, Real* rec,
                                  int& ovf, int& end) {
    Real* blk = rec + CMC_HEAD + 2 * CMC_SLOTS * f;
    int U = 0;
    for (int c = 0; c < n; ++c)
        if (c == 0 || (Real)thr[idx[c]] != (Real)thr[idx[c - 1]]) ++U;
    Real* t = blk;
    Real* T = blk + CMC_SLOTS;
    if (U >= CMC_SLOTS) {
        // too many for the block: [offset, U] in it, the values in the overflow area
        ovf |= 1 << f;
        put_int_as(blk, end);
        put_int_as(blk + 1, U);
        t = rec + end;
        T = t + U;
        end += 2 * U + 1;
    }
    double pre = 0.0;
    int u = 0;
    for (int c = 0; c < n; ++c) {
        const Real v = (Real)thr[idx[c]];
        if (c == 0 || v != (Real)thr[idx[c - 1]]) {
            t[u] = v;
            T[u] = (Real)(2.0 * pre - tot);
            ++u;
        }
        pre += alpha[idx[c]] * pol[idx[c]];
    }
    T[U] = (Real)(2.0 * pre - tot);
    if (U < CMC_SLOTS) {
        for (int i = U; i < CMC_SLOTS; ++i) t[i] = (Real)INFINITY;
        for (int i = U + 1; i < CMC_SLOTS; ++i) T[i] = T[U];
    }
}

__device__ void stage_cmc_one(int nF, int ns, const int* feat, const double* thr, const int* pol,
                              const double* alpha, int rec_len, float* rf, double* rd) {
    for (int i = 0; i < rec_len; ++i) { rf[i] = 0.f; rd[i] = 0.0; }
    double F0 = 0.0;
    for (int i = 0; i < ns; ++i)
        if (isinf(thr[i]) && thr[i] < 0) F0 += alpha[i] * pol[i];
    rf[0] = (float)F0;
    rd[0] = F0;
    int ovf_f = 0, ovf_d = 0;
    int end_f = CMC_HEAD + 2 * CMC_SLOTS * nF, end_d = end_f;
    for (int f = 0; f < nF; ++f) {
        // the feature's stumps (constant ones excluded) sorted by threshold, stable
        int idx[BAP_MAX_STUMPS];
        int n = 0;
        for (int i = 0; i < ns; ++i)
            if (feat[i] == f && !(isinf(thr[i]) && thr[i] < 0)) {
                int k = n++;
                while (k > 0 && thr[idx[k - 1]] > thr[i]) { idx[k] = idx[k - 1]; --k; }
                idx[k] = i;
            }
        double tot = 0.0;
        for (int i = 0; i < n; ++i) tot += alpha[idx[i]] * pol[idx[i]];
        stage_cmc_feature<float>(f, n, idx, thr, pol, alpha, tot, rf, ovf_f, end_f);
        stage_cmc_feature<double>(f, n, idx, thr, pol, alpha, tot, rd, ovf_d, end_d);
    }
    put_int_as(rf + 1, ovf_f);
    put_int_as(rd + 1, ovf_d);
}

__global__ void stage_cmc_kernel(int n_dates, int nF, int max_stumps, const int* n_stumps,
                                 const int* feat, const double* thr, const int* pol,
                                 const double* alpha, int rec_len, float* rec_f, double* rec_d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n_dates) return;
    const size_t o = (size_t)k * max_stumps;
    stage_cmc_one(nF, n_stumps[k], feat + o, thr + o, pol + o, alpha + o, rec_len,
                  rec_f + (size_t)k * rec_len, rec_d + (size_t)k * rec_len);
}

// ---------------------------------------------------------------------------------------------
// [class] Discrete AdaBoost on stumps for date m, one block (Section 3.2 names AdaBoost).
// Features: the d prices and Phi.  Candidates per feature, in order: the constant stump
// (threshold below every value; polarity +1 then -1), then the midpoints between consecutive
// distinct sorted values (polarity +1 then -1); with e_min the least weighted error the first
// candidate with error <= e_min + 1e-12 wins.  alpha = 1/2 ln((1-eps)/eps) with eps clamped to
// [1e-10, 1-1e-10]; stop before a stump with eps >= 1/2 and after a perfect one.
//
// The weights are FP64; the weighted errors are summed exactly in 64-bit fixed point (w 2^60,
// integer adds on the full-rate ALU instead of the narrow FP64 pipe), as one block-wide prefix
// scan per feature over contiguous segments of the sorted order.  The update is the closed form
// of the normalised step w exp(-alpha y h) / Z: w / (2 (1 - eps)) for a point the stump
// classifies right, w / (2 eps) for one it gets wrong (with that alpha the right points keep
// half of the weight).  No sum enters it, so every form of the fit gives the same weights; the
// three quotients are taken on three warps, and alpha's log once per stump at the end.

constexpr double kFix = 1152921504606846976.0;   // 2^60

// round(v * 2^60) to the nearest integer, ties to even, for 0 <= v <= 1: the same value as
// __double2ll_rn(v * 2^60) (the product is exact), from the bits of v with integer operations
// only.  v = s * 2^(e - 1075) with the 53-bit significand s, so v * 2^60 = s * 2^(e - 1015).
__device__ __forceinline__ long long fix60(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;                                  // zero or subnormal: rounds to 0
    const unsigned long long s = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = 1015 - e;                               // right shift of s
    if (sh <= 0) return (long long)(s << (-sh));           // exact (v >= 2^-7: sh >= -8)
    if (sh >= 64) return 0;                                // below 2^-64 of a unit: 0
    const unsigned long long q = s >> sh;
    const unsigned long long rem = s & ((1ull << sh) - 1);
    const unsigned long long half = 1ull << (sh - 1);
    return (long long)(q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0));
}

// Block-wide exclusive scan of two 64-bit values per thread (1024 threads); returns the block
// totals through tot_a / tot_b.  Uses red_a / red_b (32 entries each) in shared memory.
__device__ inline void block_scan2(long long& a, long long& b, long long* red_a, long long* red_b,
                                   long long& tot_a, long long& tot_b) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long ia = a, ib = b;
    for (int off = 1; off < 32; off <<= 1) {
        const long long ta = __shfl_up_sync(FULL, ia, off);
        const long long tb = __shfl_up_sync(FULL, ib, off);
        if (lane >= off) { ia += ta; ib += tb; }
    }
    if (lane == 31) { red_a[wid] = ia; red_b[wid] = ib; }
    __syncthreads();
    if (wid == 0) {
        long long xa = lane < nw ? red_a[lane] : 0, xb = lane < nw ? red_b[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const long long ta = __shfl_up_sync(FULL, xa, off);
            const long long tb = __shfl_up_sync(FULL, xb, off);
            if (lane >= off) { xa += ta; xb += tb; }
        }
        red_a[lane] = xa;     // inclusive prefix of the warp totals
        red_b[lane] = xb;
    }
    __syncthreads();
    const long long base_a = wid > 0 ? red_a[wid - 1] : 0, base_b = wid > 0 ? red_b[wid - 1] : 0;
    tot_a = red_a[nw - 1];
    tot_b = red_b[nw - 1];
    a = base_a + ia - a;      // exclusive
    b = base_b + ib - b;
    __syncthreads();
}

__device__ inline long long block_min_ll(long long v, long long* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_down_sync(0xffffffffu, v, off));
    if (lane == 0) red[wid] = v;
    __syncthreads();
    long long r = LLONG_MAX;
    for (int k = 0; k < nw; ++k) r = min(r, red[k]);
    __syncthreads();
    return r;
}

// Feature f of training point i: the d prices, then the payoff Phi in FP64 (the same
// definition as the label epilogue of the path kernel).
__device__ inline double cmc_feature(const DevModel* M, const double* X, int i, int f) {
    const int d = M->d;
    if (f < d) return X[(size_t)i * d + f];
    const double* S = X + (size_t)i * d;
    double v;
    if (M->payoff == BAP_MAX_CALL) {
        double mx = S[0];
        for (int q = 1; q < d; ++q) mx = S[q] > mx ? S[q] : mx;
        v = mx - M->K;
    } else if (M->payoff == BAP_BASKET_PUT) {
        double b = 0;
        for (int q = 0; q < d; ++q) b += M->w[q] * S[q];
        v = M->K - b;
    } else {
        double lg = 0;
        for (int q = 0; q < d; ++q) lg += M->w[q] * log(S[q]);
        v = exp(lg) - M->K;
    }
    return v > 0 ? v : 0;
}

// Order-preserving map of a double's bits to an unsigned 64-bit integer (no NaN): the sign bit
// set for values >= 0, every bit flipped for negative ones; -0 is taken as +0.  Integer compares
// run on the integer pipe, where FP64 compares would queue for the narrow FP64 one.
__device__ __forceinline__ unsigned long long ordered_from_bits(unsigned long long b) {
    if ((b << 1) == 0) b = 0;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ unsigned long long bits_from_ordered(unsigned long long k) {
    return (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
}

// One compare-exchange of the bitonic network: pair q of the stage (size, stride) joins entries
// i and i + stride, i = q with a zero bit inserted at the stride, ascending where bit `size` of
// i is clear.  Keys compare as (ordered value, index).
__device__ __forceinline__ void bitonic_cmpx(unsigned long long* k, int* idx, int q, int stride,
                                             int size) {
    const int i = ((q & ~(stride - 1)) << 1) | (q & (stride - 1));
    const int jx = i + stride;
    const bool up = (i & size) == 0;
    const unsigned long long a = k[i], b = k[jx];
    const int ia = idx[i], ib = idx[jx];
    const bool lt = b < a || (b == a && ib < ia);
    if (lt == up) {
        k[i] = b; k[jx] = a;
        idx[i] = ib; idx[jx] = ia;
    }
}

// Bitonic sort of (key, idx) pairs over P2 entries in shared memory, by (value, index), on the
// ordered integer images of the values (the doubles are restored in place at the end).  A stage
// whose pairs all lie inside one warp's chunk of P2 / warps entries runs under a warp barrier
// only; a block barrier comes before the next stage that crosses chunks.
__device__ inline void block_bitonic(double* key, int* idx, int P2) {
    unsigned long long* k = reinterpret_cast<unsigned long long*>(key);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int i = tid; i < P2; i += blockDim.x) k[i] = ordered_from_bits(k[i]);
    __syncthreads();
    const int half = P2 >> 1;
    const int chunk = P2 >= 2 * nwarps ? P2 / nwarps : 0;    // powers of two
    bool pending = false;                                   // warp-local stages since a block barrier
    for (int size = 2; size <= P2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (chunk > 0 && 2 * stride <= chunk) {
                const int q0 = warp * (chunk >> 1), q1 = q0 + (chunk >> 1);
                for (int q = q0 + lane; q < q1; q += 32) bitonic_cmpx(k, idx, q, stride, size);
                __syncwarp();
                pending = true;
            } else {
                if (pending) {
                    __syncthreads();
                    pending = false;
                }
                for (int q = tid; q < half; q += blockDim.x) bitonic_cmpx(k, idx, q, stride, size);
                __syncthreads();
            }
        }
    }
    if (pending) __syncthreads();
    for (int i = tid; i < P2; i += blockDim.x) k[i] = bits_from_ordered(k[i]);
    __syncthreads();
}

__global__ void __launch_bounds__(1024) adaboost_kernel(
    const DevModel* M, int m, int J, const double* X, const double* label_y, const int* label,
    int n_rounds, double* sorted_v, int* sorted_i, double* err, int max_stumps, int* n_stumps,
    int* feat, double* thr, int* pol, double* alpha, int rec_len, float* rec_f, double* rec_d,
    int* fitted) {
    extern __shared__ __align__(16) unsigned char smem[];
    (void)label_y;
    const int d = M->d;
    const int nF = d + 1;
    int P2 = 1;
    while (P2 < J) P2 <<= 1;
    double* w = reinterpret_cast<double*>(smem);                         // J
    unsigned char* region = smem + (size_t)J * 8;                        // sort keys, then wf
    double* key = reinterpret_cast<double*>(region);                     // P2 (sorting only)
    int* idx = reinterpret_cast<int*>(key + P2);                         // P2 (sorting only)
    long long* wf = reinterpret_cast<long long*>(region);                // J (rounds only)
    const size_t region_bytes = (size_t)P2 * 12 > (size_t)J * 8 ? (size_t)P2 * 12 : (size_t)J * 8;
    signed char* lab = reinterpret_cast<signed char*>(region + region_bytes);   // J
    long long* errl = reinterpret_cast<long long*>(err);                 // nF x J, -1 = no split
    __shared__ long long red_a[32], red_b[32], red_m[32];
    __shared__ long long s_neg[MAXF];
    __shared__ double s_thr, s_fok, s_fbad;
    __shared__ int s_f, s_pol, s_stop, s_count;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // sort each feature (bitonic on (value, index)); the payoff feature is Phi in FP64 (the same
    // definition as the label epilogue of the path kernel)
    for (int f = 0; f < nF; ++f) {
        for (int i = tid; i < P2; i += blockDim.x) {
            key[i] = i < J ? cmc_feature(M, X, i, f) : INFINITY;
            idx[i] = i < J ? i : 0x7fffffff;
        }
        __syncthreads();
        block_bitonic(key, idx, P2);
        for (int i = tid; i < J; i += blockDim.x) {
            sorted_v[(size_t)f * J + i] = key[i];
            sorted_i[(size_t)f * J + i] = idx[i];
        }
        __syncthreads();
    }
    for (int i = tid; i < J; i += blockDim.x) {
        w[i] = 1.0 / (double)J;
        lab[i] = label[i] > 0 ? 1 : -1;
    }
    if (tid == 0) s_count = 0;
    __syncthreads();

    // contiguous segment of the sorted order per thread
    const int per = (J + blockDim.x - 1) / blockDim.x;
    const int lo = tid * per, hi = min(J, lo + per);
    const long long tol = (long long)(1e-12 * kFix);
    const size_t o_st = (size_t)m * max_stumps;
    for (int round = 0; round < n_rounds; ++round) {
        // fixed-point weights and their total
        long long part = 0;
        for (int i = tid; i < J; i += blockDim.x) {
            const long long v = fix60(w[i]);
            wf[i] = v;
            part += v;
        }
        long long Wp = part, dummy = 0, Wtot = 0, dtot = 0;
        block_scan2(Wp, dummy, red_a, red_b, Wtot, dtot);
        const long long W = Wtot;
        // pass 1: errors of every candidate, least error per feature
        long long emin = LLONG_MAX;
        for (int f = 0; f < nF; ++f) {
            const int* six = sorted_i + (size_t)f * J;
            const double* sv = sorted_v + (size_t)f * J;
            long long sp = 0, sn = 0;
            for (int i = lo; i < hi; ++i) {
                const int k = six[i];
                if (lab[k] > 0) sp += wf[k]; else sn += wf[k];
            }
            long long pp = sp, pn = sn, tot_p = 0, tot_n = 0;
            block_scan2(pp, pn, red_a, red_b, tot_p, tot_n);
            const long long neg = tot_n;
            if (tid == 0) s_neg[f] = neg;
            long long my = min(neg, W - neg);
            for (int i = lo; i < hi; ++i) {
                const int k = six[i];
                if (lab[k] > 0) pp += wf[k]; else pn += wf[k];
                long long e = -1;
                if (i < J - 1 && sv[i + 1] > sv[i]) {
                    e = pp + (neg - pn);
                    my = min(my, min(e, W - e));
                }
                if (i < J - 1) errl[(size_t)f * J + i] = e;
            }
            emin = min(emin, my);
        }
        emin = block_min_ll(emin, red_m);
        const long long lim = emin + tol;
        // pass 2: the first candidate (feature, threshold, polarity order) within the tolerance
        long long chosen = LLONG_MAX;
        int cf = -1;
        for (int f = 0; f < nF && cf < 0; ++f) {
            const long long neg = s_neg[f];
            long long c = LLONG_MAX;
            if (neg <= lim) c = 0;
            else if (W - neg <= lim) c = 1;
            else {
                for (int i = lo; i < hi && c == LLONG_MAX; ++i) {
                    if (i >= J - 1) break;
                    const long long e = errl[(size_t)f * J + i];
                    if (e < 0) continue;
                    if (e <= lim) c = 2 + 2LL * i;
                    else if (W - e <= lim) c = 3 + 2LL * i;
                }
            }
            c = block_min_ll(c, red_m);
            if (c != LLONG_MAX) { chosen = c; cf = f; }
        }
        // the decision: lane 0 of warps 0, 1 and 2 (warp 0 the stopping rule and the record,
        // warps 1 and 2 one update factor each)
        if (lane == 0 && warp < 3) {
            const int f = cf < 0 ? 0 : cf;
            const long long c = cf < 0 ? 0 : chosen;
            long long e;
            int pl;
            int i = 0;
            if (c < 2) {
                pl = c == 0 ? 1 : -1;
                e = c == 0 ? s_neg[f] : W - s_neg[f];
            } else {
                i = (int)((c - 2) / 2);
                pl = ((c - 2) % 2 == 0) ? 1 : -1;
                const long long ep = errl[(size_t)f * J + i];
                e = pl > 0 ? ep : W - ep;
            }
            if (cf < 0) e = W;                          // no candidate at all: stop below
            if (warp == 0) {
                const double eps = (double)e / (double)W;
                s_stop = 0;
                if (eps >= 0.5 - 1e-12) {
                    s_stop = 1;
                } else {
                    const double th = c < 2 ? -INFINITY
                                            : 0.5 * (sorted_v[(size_t)f * J + i] + sorted_v[(size_t)f * J + i + 1]);
                    const int k = s_count++;
                    feat[o_st + k] = f;
                    thr[o_st + k] = th;
                    pol[o_st + k] = pl;
                    alpha[o_st + k] = fmin(fmax(eps, 1e-10), 1.0 - 1e-10);   // log at the end
                    s_f = f; s_thr = th; s_pol = pl;
                    if (eps <= 1e-10) s_stop = 2;
                }
            } else if (warp == 1) {
                s_fok = (0.5 * (double)W) / (double)(W - e);
            } else {
                s_fbad = (0.5 * (double)W) / (double)e;
            }
        }
        __syncthreads();
        if (s_stop != 0) break;
        // the normalised update in closed form: 1 / (2 (1 - eps)) for a point the stump
        // classifies right, 1 / (2 eps) for one it gets wrong
        {
            const int f = s_f;
            const double th = s_thr, fok = s_fok, fbad = s_fbad;
            const int pl = s_pol;
            const double* sv = sorted_v + (size_t)f * J;
            const int* six = sorted_i + (size_t)f * J;
            for (int r = tid; r < J; r += blockDim.x) {
                const int i = six[r];
                const int h = sv[r] > th ? pl : -pl;
                w[i] *= (h == lab[i] ? fok : fbad);
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int k = tid; k < s_count; k += blockDim.x) {
        const double ec = alpha[o_st + k];
        alpha[o_st + k] = 0.5 * log((1.0 - ec) / ec);
    }
    __syncthreads();
    if (tid == 0) {
        n_stumps[m] = s_count;
        stage_cmc_one(nF, s_count, feat + o_st, thr + o_st, pol + o_st, alpha + o_st, rec_len,
                      rec_f + (size_t)m * rec_len, rec_d + (size_t)m * rec_len);
        fitted[m] = 1;
    }
}

// ---------------------------------------------------------------------------------------------
// [class] The same AdaBoost fit on a thread-block cluster: block f (cluster rank f) owns feature
// f, so the per-feature sorts, prefix scans and error searches of a round run on nF SMs at once.
// Every block keeps its own copy of the weights and applies the same update, so the copies
// stay identical.  Per round the blocks exchange, through the distributed shared
// memory of the leader block (rank 0): the least error of each feature, then the first
// candidate of each feature within the tolerance and its error and threshold.  Two cluster
// barriers per round; every decision is taken from values read back from the leader, so all
// blocks take the same branches and meet the same barriers.  Choices, tie rule and update are
// those of adaboost_kernel.

struct BoostExchange {
    long long W;                   // fixed-point total weight of the round (the leader's)
    long long fmin[MAXF];          // least error per feature
    long long cand[MAXF];          // first candidate code per feature within the tolerance
    long long cerr[MAXF];          // its error
    double cthr[MAXF];             // its threshold
};

__global__ void __launch_bounds__(kClusterBoostThreads) adaboost_cluster_kernel(
    const DevModel* M, int m, int J, const double* X, const int* label, int n_rounds,
    double* sorted_v, int* sorted_i, int max_stumps, int* n_stumps, int* feat, double* thr,
    int* pol, double* alpha, int rec_len, float* rec_f, double* rec_d, int* fitted) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const unsigned FULL = 0xffffffffu;
    const int d = M->d;
    const int nF = d + 1;
    const int f = (int)cluster.block_rank();            // the feature of this block
    int P2 = 1;
    while (P2 < J) P2 <<= 1;
    const int nwords = (J + 31) / 32;
    // shared memory: w | region (sort keys, then wf, six, inv) | lab | split | mask | cmask
    double* w = reinterpret_cast<double*>(smem);                          // J
    unsigned char* region = smem + (size_t)J * 8;
    double* key = reinterpret_cast<double*>(region);                      // P2 (sort)
    int* idx = reinterpret_cast<int*>(key + P2);                          // P2 (sort)
    long long* wf = reinterpret_cast<long long*>(region);                 // J fixed-point weights
    int* six = reinterpret_cast<int*>(region + (size_t)J * 8);           // J: sorted position -> point
    int* inv = six + J;                                                    // J: point -> sorted position
    const size_t region_bytes = (size_t)P2 * 12 > (size_t)J * 16 ? (size_t)P2 * 12 : (size_t)J * 16;
    signed char* lab = reinterpret_cast<signed char*>(region + region_bytes);   // J
    unsigned char* split = reinterpret_cast<unsigned char*>(lab + J);     // J: a threshold after r
    unsigned* mask = reinterpret_cast<unsigned*>(smem + ((size_t)J * 8 + region_bytes + 2 * (size_t)J + 3) / 4 * 4);
    unsigned* cmask = mask + nwords;                                       // the chosen stump's
    __shared__ BoostExchange ex;                         // read remotely on the leader only
    __shared__ long long red_a[32], red_b[32];
    __shared__ long long s_min, s_cand, s_lim, s_W;
    __shared__ double s_thr, s_ec, s_cok, s_cbad;
    __shared__ int s_f, s_pol, s_stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    BoostExchange* lead = cluster.map_shared_rank(&ex, 0);

    // sort this block's feature and publish it; keep the permutation both ways, and where the
    // sorted values step (a threshold can sit after position r), in shared memory
    for (int i = tid; i < P2; i += blockDim.x) {
        key[i] = i < J ? cmc_feature(M, X, i, f) : INFINITY;
        idx[i] = i < J ? i : 0x7fffffff;
    }
    __syncthreads();
    block_bitonic(key, idx, P2);
    for (int r = tid; r < J; r += blockDim.x) {
        sorted_v[(size_t)f * J + r] = key[r];
        sorted_i[(size_t)f * J + r] = idx[r];
        split[r] = (r < J - 1 && key[r + 1] > key[r]) ? 1 : 0;
    }
    __syncthreads();
    for (int r = tid; r < J; r += blockDim.x) {
        const int k = sorted_i[(size_t)f * J + r];
        six[r] = k;
        inv[k] = r;
    }
    for (int i = tid; i < J; i += blockDim.x) {
        w[i] = 1.0 / (double)J;
        wf[i] = fix60(w[i]);
        lab[i] = label[i] > 0 ? 1 : -1;
    }
    __threadfence();          // the sorted features are read by every block of the cluster
    cluster.sync();

    const int per = (J + blockDim.x - 1) / blockDim.x;
    const int lo = tid * per, hi = min(J, lo + per);
    const long long tol = (long long)(1e-12 * kFix);
    const size_t o_st = (size_t)m * max_stumps;
    int count = 0;
    for (int round = 0; round < n_rounds; ++round) {
        if (tid == 0) s_min = LLONG_MAX;
        // prefix of this feature's positive and negative weights over the sorted order; the two
        // totals give the round's total weight exactly
        long long sp = 0, sn = 0;
        for (int r = lo; r < hi; ++r) {
            const int k = six[r];
            if (lab[k] > 0) sp += wf[k]; else sn += wf[k];
        }
        long long pp0 = sp, pn0 = sn, tot_p = 0, tot_n = 0;
        block_scan2(pp0, pn0, red_a, red_b, tot_p, tot_n);
        const long long W = tot_p + tot_n;
        const long long neg = tot_n;
        long long my = min(neg, W - neg);
        {
            long long pp = pp0, pn = pn0;
            for (int r = lo; r < hi; ++r) {
                const int k = six[r];
                if (lab[k] > 0) pp += wf[k]; else pn += wf[k];
                if (split[r]) {
                    const long long e = pp + (neg - pn);
                    my = min(my, min(e, W - e));
                }
            }
        }
        atomicMin(&s_min, my);
        __syncthreads();
        if (tid == 0) {
            lead->fmin[f] = s_min;
            if (f == 0) ex.W = W;
        }
        cluster.sync();
        // the first candidate of this feature within the tolerance of the overall least error
        if (tid == 0) {
            long long emin = LLONG_MAX;
            for (int g = 0; g < nF; ++g) emin = min(emin, lead->fmin[g]);
            s_lim = emin + tol;
            s_W = lead->W;
            s_cand = LLONG_MAX;
        }
        __syncthreads();
        const long long Wl = s_W;
        const long long lim = s_lim;
        long long c = LLONG_MAX;
        if (neg <= lim) c = 0;
        else if (W - neg <= lim) c = 1;
        else {
            long long pp = pp0, pn = pn0;
            for (int r = lo; r < hi && c == LLONG_MAX; ++r) {
                const int k = six[r];
                if (lab[k] > 0) pp += wf[k]; else pn += wf[k];
                if (!split[r]) continue;
                const long long e = pp + (neg - pn);
                if (e <= lim) c = 2 + 2LL * r;
                else if (W - e <= lim) c = 3 + 2LL * r;
            }
        }
        if (c != LLONG_MAX) atomicMin(&s_cand, c);
        __syncthreads();
        const long long cmin = s_cand;
        if (cmin < 2 || cmin == LLONG_MAX ? tid == 0 : c == cmin) {
            // thread 0 for a constant stump or no candidate; else the one thread whose
            // segment holds the threshold
            long long e = 0;
            double th = -INFINITY;
            if (cmin == 0) e = neg;
            else if (cmin == 1) e = W - neg;
            else if (cmin != LLONG_MAX) {
                const int r0 = (int)((cmin - 2) / 2);
                long long pp = pp0, pn = pn0;
                for (int r = lo; r <= r0; ++r) {
                    const int k = six[r];
                    if (lab[k] > 0) pp += wf[k]; else pn += wf[k];
                }
                const long long ep = pp + (neg - pn);
                e = ((cmin - 2) % 2 == 0) ? ep : W - ep;
                th = 0.5 * (sorted_v[(size_t)f * J + r0] + sorted_v[(size_t)f * J + r0 + 1]);
            }
            lead->cand[f] = cmin;
            lead->cerr[f] = e;
            lead->cthr[f] = th;
        }
        // which points lie above this feature's candidate threshold, one bit per point (read by
        // every block if this feature's stump is chosen)
        {
            const int rstar = cmin >= 2 && cmin != LLONG_MAX ? (int)((cmin - 2) / 2) : -1;
            for (int wd = warp; wd < nwords; wd += nwarps) {
                const int i = wd * 32 + lane;
                const bool above = i < J && inv[i] > rstar;
                const unsigned bits = __ballot_sync(FULL, above);
                if (lane == 0) mask[wd] = bits;
            }
        }
        cluster.sync();
        // the chosen stump: the first feature with a candidate.  Lane 0 of warps 0, 1 and 2 of
        // every block read the same leader values and take the same decision (warp 0 the
        // stopping rule, warps 1 and 2 one update factor each, on three sub-partitions)
        if (lane == 0 && warp < 3) {
            int cf = -1;
            long long cc = 0;
            for (int g = 0; g < nF && cf < 0; ++g) {
                const long long v = lead->cand[g];
                if (v != LLONG_MAX) { cf = g; cc = v; }
            }
            const long long e = cf < 0 ? Wl : lead->cerr[cf];     // no candidate at all: stop below
            if (warp == 0) {
                const double eps = (double)e / (double)Wl;
                s_stop = 0;
                if (eps >= 0.5 - 1e-12) {
                    s_stop = 1;
                } else {
                    s_f = cf;
                    s_thr = lead->cthr[cf];
                    s_pol = (cc < 2) ? (cc == 0 ? 1 : -1) : (((cc - 2) % 2 == 0) ? 1 : -1);
                    s_ec = fmin(fmax(eps, 1e-10), 1.0 - 1e-10);
                    if (eps <= 1e-10) s_stop = 2;
                }
            } else if (warp == 1) {
                s_cok = (0.5 * (double)Wl) / (double)(Wl - e);
            } else {
                s_cbad = (0.5 * (double)Wl) / (double)e;
            }
        }
        __syncthreads();
        if (s_stop == 1) break;
        const int fs = s_f;
        const int pl = s_pol;
        if (f == 0 && tid == 0) {
            feat[o_st + count] = fs;
            thr[o_st + count] = s_thr;
            pol[o_st + count] = pl;
            alpha[o_st + count] = s_ec;                 // 1/2 ln((1 - eps) / eps) at the end
        }
        ++count;
        if (s_stop == 2) break;
        {
            const unsigned* src = cluster.map_shared_rank(mask, fs);
            for (int wd = tid; wd < nwords; wd += blockDim.x) cmask[wd] = src[wd];
        }
        __syncthreads();
        // the normalised update in closed form (1 / (2 (1 - eps)) right, 1 / (2 eps) wrong) and
        // the next round's fixed-point weights; no sum enters, so every block's copy is the same
        {
            const double cok = s_cok, cbad = s_cbad;
            for (int i = tid; i < J; i += blockDim.x) {
                const int h = ((cmask[i >> 5] >> (i & 31)) & 1u) ? pl : -pl;
                const double v = w[i] * (h == lab[i] ? cok : cbad);
                w[i] = v;
                wf[i] = fix60(v);
            }
            __syncthreads();
        }
    }
    if (f == 0) {
        for (int k = tid; k < count; k += blockDim.x) {
            const double ec = alpha[o_st + k];
            alpha[o_st + k] = 0.5 * log((1.0 - ec) / ec);
        }
        __syncthreads();
        if (tid == 0) {
            n_stumps[m] = count;
            stage_cmc_one(nF, count, feat + o_st, thr + o_st, pol + o_st, alpha + o_st, rec_len,
                          rec_f + (size_t)m * rec_len, rec_d + (size_t)m * rec_len);
            fitted[m] = 1;
        }
    }
    cluster.sync();           // the leader's exchange area and the masks stay until all are done
}

// ---------------------------------------------------------------------------------------------
// [class] The same AdaBoost fit in one 512-thread block, one warp per feature.  A feature's
// sorted order sits in shared memory as 16-bit point indices (the top bit marks a position after
// which a threshold can sit) and the weights as signed fixed-point values s_i = lab_i wf_i in
// point order.  The error of polarity +1 at split r of feature f is neg_f + S_f(r), S_f the
// prefix of s along f's order, so a round costs the warp of f one gather per position.  Lane l
// owns positions 32 l .. 32 l + 31 of every 1024, stored transposed so that the warp's loads are
// conflict free; per segment of 32 the warp keeps the prefix at its start and the least and
// largest prefix at a split.  Those give the feature's least error, min(neg + min S,
// W - neg - max S), and, once the round's least error is known, the first segment holding a
// candidate, which the whole warp rescans.  Choices, tie rule and weight update are those of
// adaboost_cluster_kernel, so the stumps are the cluster form's bit for bit; the round's three
// FP64 quotients run on three warps and the thresholds and logs once per stump at the end.

// Storage index of sorted position r (and, the map being its own inverse, the position held at
// storage index r): the two 5-bit fields below bit 10 swapped.
__device__ __forceinline__ int warp_boost_tpos(int r) {
    return (r & ~1023) | ((r & 31) << 5) | ((r >> 5) & 31);
}

__global__ void __launch_bounds__(kWarpBoostThreads) adaboost_warp_kernel(
    const DevModel* M, int m, int J, const double* X, const int* label, int n_rounds,
    double* sorted_v, int* sorted_i, int max_stumps, int* n_stumps, int* feat, double* thr,
    int* pol, double* alpha, int rec_len, float* rec_f, double* rec_d, int* fitted) {
    extern __shared__ __align__(16) unsigned char smem[];
    const unsigned FULL = 0xffffffffu;
    constexpr int nthr = kWarpBoostThreads;
    const int d = M->d;
    const int nF = d + 1;
    int P2 = 1;
    while (P2 < J) P2 <<= 1;
    const int nsc = (J + 1023) >> 10;              // blocks of 1024 sorted positions
    const int NP = nsc << 10;                      // stored positions per feature
    const int nseg = nF * nsc * 32;
    // shared memory: region (sort keys, then w | s) | pos | segment base, min, max | lab
    const size_t ra = warp_boost_region(J);
    double* key = reinterpret_cast<double*>(smem);                        // P2 (sorting only)
    int* idx = reinterpret_cast<int*>(key + P2);                          // P2 (sorting only)
    double* w = reinterpret_cast<double*>(smem);                          // J FP64 weights
    long long* sw = reinterpret_cast<long long*>(smem + (size_t)J * 8);  // J + 1 (s_J = 0: padding)
    unsigned short* pos = reinterpret_cast<unsigned short*>(smem + ra);   // nF x NP
    long long* sg_base = reinterpret_cast<long long*>(smem + ra + (size_t)nF * NP * 2);
    long long* sg_min = sg_base + nseg;
    long long* sg_max = sg_min + nseg;
    signed char* lab = reinterpret_cast<signed char*>(sg_max + nseg);    // J
    __shared__ long long s_fmin[MAXF], s_fneg[MAXF], s_cand[MAXF], s_cerr[MAXF];
    __shared__ double s_cthr[MAXF];
    __shared__ unsigned long long s_W;
    __shared__ double s_cok, s_cbad, s_Wd, s_hWd;
    __shared__ int s_f, s_pol, s_stop, s_rstar;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // sort every feature (bitonic on (value, index), the whole block per feature); publish it
    // and keep its order, with the split marks, in shared memory
    for (int f = 0; f < nF; ++f) {
        for (int i = tid; i < P2; i += nthr) {
            key[i] = i < J ? cmc_feature(M, X, i, f) : INFINITY;
            idx[i] = i < J ? i : 0x7fffffff;
        }
        __syncthreads();
        block_bitonic(key, idx, P2);
        for (int r = tid; r < NP; r += nthr) {
            unsigned short u = (unsigned short)J;          // padding: the zero-weight point J
            if (r < J) {
                sorted_v[(size_t)f * J + r] = key[r];
                sorted_i[(size_t)f * J + r] = idx[r];
                // (a padding index can only sort below J if a feature were NaN: it then maps to
                // the zero-weight point J, so no access leaves the arrays)
                const int k = idx[r] < J ? idx[r] : J;
                u = (unsigned short)(k | ((r < J - 1 && key[r + 1] > key[r]) ? 0x8000 : 0));
            }
            pos[(size_t)f * NP + warp_boost_tpos(r)] = u;
        }
        __syncthreads();
    }
    const long long w0 = fix60(1.0 / (double)J);
    for (int i = tid; i < J; i += nthr) {
        w[i] = 1.0 / (double)J;
        const signed char l = label[i] > 0 ? 1 : -1;
        lab[i] = l;
        sw[i] = l > 0 ? w0 : -w0;
    }
    if (tid == 0) {
        sw[J] = 0;
        s_W = (unsigned long long)(w0 * (long long)J);
        s_stop = 0;
    }
    __syncthreads();

    const long long tol = (long long)(1e-12 * kFix);
    const size_t o_st = (size_t)m * max_stumps;
    int count = 0;
    for (int round = 0; round < n_rounds; ++round) {
        const long long W = (long long)s_W;            // exact total of the fixed-point weights
        // the round's W in FP64 for the decision, off its path (the last warp owns no feature)
        if (tid == nthr - 32) {
            s_Wd = (double)W;
            s_hWd = 0.5 * (double)W;
        }
        // pass 1 (warp f): prefix sums along feature f's order; the negatives' total follows
        // from W and the signed total
        if (warp < nF) {
            const int f = warp;
            const unsigned short* P = pos + (size_t)f * NP;
            long long carry = 0, amin = LLONG_MAX, amax = LLONG_MIN;
            for (int sc = 0; sc < nsc; ++sc) {
                const unsigned short* Q = P + (sc << 10) + lane;
                long long T = 0, tmin = LLONG_MAX, tmax = LLONG_MIN;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const unsigned u = Q[j << 5];
                    T += sw[u & 0x7fffu];
                    if (u & 0x8000u) {
                        tmin = min(tmin, T);
                        tmax = max(tmax, T);
                    }
                }
                long long incl = T;
                for (int off = 1; off < 32; off <<= 1) {
                    const long long t = __shfl_up_sync(FULL, incl, off);
                    if (lane >= off) incl += t;
                }
                const long long base = carry + incl - T;
                carry += __shfl_sync(FULL, incl, 31);
                const long long smn = tmin == LLONG_MAX ? LLONG_MAX : base + tmin;
                const long long smx = tmax == LLONG_MIN ? LLONG_MIN : base + tmax;
                const int s = (f * nsc + sc) * 32 + lane;
                sg_base[s] = base;
                sg_min[s] = smn;
                sg_max[s] = smx;
                amin = min(amin, smn);
                amax = max(amax, smx);
            }
            for (int off = 16; off > 0; off >>= 1) {
                amin = min(amin, __shfl_xor_sync(FULL, amin, off));
                amax = max(amax, __shfl_xor_sync(FULL, amax, off));
            }
            const long long neg = (W - carry) / 2;      // W - S = 2 (negatives' weight), exact
            long long mn = min(neg, W - neg);
            if (amin != LLONG_MAX) mn = min(mn, neg + amin);
            if (amax != LLONG_MIN) mn = min(mn, W - (neg + amax));
            if (lane == 0) {
                s_fmin[f] = mn;
                s_fneg[f] = neg;
            }
        }
        __syncthreads();
        // pass 2 (warp f): the first candidate of feature f within the tolerance of the least
        // error over all features
        if (warp < nF) {
            const int f = warp;
            long long emin = LLONG_MAX;
            for (int g = 0; g < nF; ++g) emin = min(emin, s_fmin[g]);
            const long long lim = emin + tol;
            const long long neg = s_fneg[f];
            long long c = LLONG_MAX, e = 0;
            int r0 = -1;
            if (neg <= lim) {
                c = 0;
                e = neg;
            } else if (W - neg <= lim) {
                c = 1;
                e = W - neg;
            } else {
                for (int sc = 0; sc < nsc && c == LLONG_MAX; ++sc) {
                    const int s0 = (f * nsc + sc) * 32;
                    const long long smn = sg_min[s0 + lane], smx = sg_max[s0 + lane];
                    const bool hit = (smn != LLONG_MAX && neg + smn <= lim) ||
                                     (smx != LLONG_MIN && W - (neg + smx) <= lim);
                    const unsigned b = __ballot_sync(FULL, hit);
                    if (!b) continue;
                    // the first such segment, rescanned by the warp: lane j takes its position j
                    const int L = __ffs(b) - 1;
                    const unsigned u = pos[(size_t)f * NP + (sc << 10) + (lane << 5) + L];
                    long long incl = sw[u & 0x7fffu];
                    for (int off = 1; off < 32; off <<= 1) {
                        const long long t = __shfl_up_sync(FULL, incl, off);
                        if (lane >= off) incl += t;
                    }
                    const long long er = neg + sg_base[s0 + L] + incl;
                    const bool q = (u & 0x8000u) && (er <= lim || W - er <= lim);
                    const unsigned bq = __ballot_sync(FULL, q);
                    if (!bq) continue;                     // not reached: the segment holds one
                    const int j = __ffs(bq) - 1;
                    const long long ej = __shfl_sync(FULL, er, j);
                    r0 = (sc << 10) + (L << 5) + j;
                    if (ej <= lim) {
                        c = 2 + 2LL * r0;
                        e = ej;
                    } else {
                        c = 3 + 2LL * r0;
                        e = W - ej;
                    }
                }
            }
            if (lane == 0) {
                s_cand[f] = c;
                s_cerr[f] = e;
                s_cthr[f] = r0 >= 0 ? (double)r0 : -INFINITY;    // the position; value at the end
            }
        }
        __syncthreads();
        // the chosen stump: the first feature with a candidate.  Lane 0 of warps 0, 1 and 2
        // (three sub-partitions) take the same decision and one FP64 quotient each: eps = e / W
        // with the stopping rule and the record, and the update factors 1 / (2 (1 - eps)) =
        // (W / 2) / (W - e) and 1 / (2 eps) = (W / 2) / e
        if (lane == 0 && warp < 3) {
            int cf = -1;
            long long cc = 0;
            for (int g = 0; g < nF && cf < 0; ++g) {
                if (s_cand[g] != LLONG_MAX) {
                    cf = g;
                    cc = s_cand[g];
                }
            }
            const long long ce = cf < 0 ? W : s_cerr[cf];     // no candidate at all: stop below
            if (warp == 0) {
                const double eps = (double)ce / s_Wd;
                s_stop = 0;
                if (eps >= 0.5 - 1e-12) {
                    s_stop = 1;
                } else {
                    const int pl0 = (cc < 2) ? (cc == 0 ? 1 : -1) : (((cc - 2) % 2 == 0) ? 1 : -1);
                    s_f = cf;
                    s_pol = pl0;
                    s_rstar = cc >= 2 ? (int)((cc - 2) / 2) : -1;
                    feat[o_st + count] = cf;
                    thr[o_st + count] = s_cthr[cf];
                    pol[o_st + count] = pl0;
                    alpha[o_st + count] = eps;                 // clamped, and its log, at the end
                    if (eps <= 1e-10) s_stop = 2;
                }
                s_W = 0ull;                                // every thread holds this round's W
            } else if (warp == 1) {
                s_cok = s_hWd / (double)(W - ce);
            } else {
                s_cbad = s_hWd / (double)ce;
            }
        }
        __syncthreads();
        if (s_stop != 0) break;
        ++count;
        // the normalised AdaBoost update in closed form: exp(-+alpha) / Z is 1 / (2 (1 - eps))
        // for a point the stump classifies right and 1 / (2 eps) for one it gets wrong.  No sum
        // enters, so the order is free: walk the chosen feature's stored order, whose position
        // tells the stump's vote
        {
            const int rstar = s_rstar, pl = s_pol;
            const double cok = s_cok, cbad = s_cbad;
            const unsigned short* P = pos + (size_t)s_f * NP;
            long long ws = 0;
            for (int k = tid; k < NP; k += nthr) {
                const int r = warp_boost_tpos(k);
                const int i = P[k] & 0x7fff;
                if (r < J && i < J) {
                    const int h = r > rstar ? pl : -pl;
                    const double v = w[i] * (h == lab[i] ? cok : cbad);
                    w[i] = v;
                    const long long q = fix60(v);
                    sw[i] = lab[i] > 0 ? q : -q;
                    ws += q;
                }
            }
            for (int off = 16; off > 0; off >>= 1) ws += __shfl_down_sync(FULL, ws, off);
            if (lane == 0) atomicAdd(&s_W, (unsigned long long)ws);
        }
        __syncthreads();
    }
    // a stump that stopped the fit with eps <= 1e-10 is kept (count it); then, one thread per
    // stump, alpha = 1/2 ln((1 - eps) / eps) and the threshold between sorted positions r, r + 1
    if (s_stop == 2) ++count;
    for (int k = tid; k < count; k += nthr) {
        const double ec = fmin(fmax(alpha[o_st + k], 1e-10), 1.0 - 1e-10);
        alpha[o_st + k] = 0.5 * log((1.0 - ec) / ec);
        const double t = thr[o_st + k];
        if (t >= 0.0) {
            const double* sv = sorted_v + (size_t)feat[o_st + k] * J;
            const int r = (int)t;
            thr[o_st + k] = 0.5 * (sv[r] + sv[r + 1]);
        }
    }
    __syncthreads();
    if (tid == 0) {
        n_stumps[m] = count;
        stage_cmc_one(nF, count, feat + o_st, thr + o_st, pol + o_st, alpha + o_st, rec_len,
                      rec_f + (size_t)m * rec_len, rec_d + (size_t)m * rec_len);
        fitted[m] = 1;
    }
}

// ---------------------------------------------------------------------------------------------
// [class] LogitBoost (Section 3.2 names it beside AdaBoost) with regression stumps on a
// thread-block cluster, block f owning feature f.  Each round: p = 1 / (1 + e^{-2F}),
// w = p (1 - p), z = (y* - p) / w clamped to [-4, 4]; the stump of largest weighted
// least-squares gain S_L^2 / W_L + S_R^2 / W_R over the splits between distinct sorted values
// (no split: S^2 / W), the first within a relative 1e-12 of the largest in (no split, feature,
// threshold) order; leaves c = S / W; F <- F + f / 2.  The sums of w and w z are exact in 2^48
// fixed point.  Block f computes p, w and z (an FP64 exp each) for its own slice of the points
// and the blocks gather each other's slices through distributed shared memory; split gains are
// screened in FP32 and taken exactly in FP64 only near the largest (see below).  A
// round is stored as two vote stumps (threshold stump |B|, constant |A|; A = (c_L + c_R) / 4,
// B = (c_R - c_L) / 4), so the rule staging and the path kernel are the AdaBoost ones.

constexpr double kLbFix = 281474976710656.0;      // 2^48
constexpr double kLbZmax = 4.0;

struct LogitExchange {
    long long W, S;                 // round totals (the leader's)
    unsigned long long gmax[MAXF];  // largest gain per feature (bit pattern of a double >= 0)
    int cand[MAXF];                 // first split position within the tolerance, -1 none
    double cthr[MAXF], ccl[MAXF], ccr[MAXF];
};

__global__ void __launch_bounds__(kClusterBoostThreads) logitboost_cluster_kernel(
    const DevModel* M, int m, int J, const double* X, const int* label, int n_rounds,
    double* sorted_v, int* sorted_i, int max_stumps, int* n_stumps, int* feat, double* thr,
    int* pol, double* alpha, int rec_len, float* rec_f, double* rec_d, int* fitted) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const unsigned FULL = 0xffffffffu;
    const int d = M->d;
    const int nF = d + 1;
    const int f = (int)cluster.block_rank();
    int P2 = 1;
    while (P2 < J) P2 <<= 1;
    const int nwords = (J + 31) / 32;
    const int ns = (J + nF - 1) / nF;                // slice of points whose p this block computes
    const int s_lo = f * ns, s_hi = min(J, s_lo + ns);
    // shared memory: F (slice) | region (sort keys, then wq, sq, six, inv) | ys | split | mask
    double* Fs = reinterpret_cast<double*>(smem);                         // ns
    unsigned char* region = smem + (size_t)ns * 8;
    double* key = reinterpret_cast<double*>(region);
    int* idx = reinterpret_cast<int*>(key + P2);
    long long* wq = reinterpret_cast<long long*>(region);                  // J
    long long* sq = wq + J;                                                 // J
    int* six = reinterpret_cast<int*>(sq + J);                             // J
    int* inv = six + J;                                                     // J
    const size_t region_bytes = (size_t)P2 * 12 > (size_t)J * 24 ? (size_t)P2 * 12 : (size_t)J * 24;
    unsigned char* ys = region + region_bytes;                              // J: y* in {0, 1}
    unsigned char* split = ys + J;                                          // J
    unsigned* mask = reinterpret_cast<unsigned*>(smem + ((size_t)ns * 8 + region_bytes + 2 * (size_t)J + 3) / 4 * 4);
    __shared__ LogitExchange ex;
    __shared__ long long red_a[32], red_b[32];
    __shared__ unsigned long long s_gmax;
    __shared__ unsigned s_gmax32;
    __shared__ int s_first, s_f, s_const, s_stop;
    __shared__ double s_lim, s_thr, s_cl, s_cr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    LogitExchange* lead = cluster.map_shared_rank(&ex, 0);

    for (int i = tid; i < P2; i += blockDim.x) {
        key[i] = i < J ? cmc_feature(M, X, i, f) : INFINITY;
        idx[i] = i < J ? i : 0x7fffffff;
    }
    __syncthreads();
    block_bitonic(key, idx, P2);
    for (int r = tid; r < J; r += blockDim.x) {
        sorted_v[(size_t)f * J + r] = key[r];
        sorted_i[(size_t)f * J + r] = idx[r];
        split[r] = (r < J - 1 && key[r + 1] > key[r]) ? 1 : 0;
    }
    __syncthreads();
    for (int r = tid; r < J; r += blockDim.x) {
        const int k = sorted_i[(size_t)f * J + r];
        six[r] = k;
        inv[k] = r;
    }
    for (int i = tid; i < J; i += blockDim.x) ys[i] = label[i] > 0 ? 1 : 0;
    for (int i = s_lo + tid; i < s_hi; i += blockDim.x) Fs[i - s_lo] = 0.0;
    __threadfence();
    cluster.sync();

    const double* sv = sorted_v + (size_t)f * J;
    const int per = (J + blockDim.x - 1) / blockDim.x;
    const int lo = tid * per, hi = min(J, lo + per);
    const size_t o_st = (size_t)m * max_stumps;
    int count = 0;
    for (int round = 0; round < n_rounds; ++round) {
        // this block's slice of w and w z in fixed point
        for (int i = s_lo + tid; i < s_hi; i += blockDim.x) {
            const double p = 1.0 / (1.0 + exp(-2.0 * Fs[i - s_lo]));
            const double w = p * (1.0 - p);
            const double z = fmin(fmax(((double)ys[i] - p) / w, -kLbZmax), kLbZmax);
            wq[i] = __double2ll_rn(w * kLbFix);
            sq[i] = __double2ll_rn((w * z) * kLbFix);
        }
        if (tid == 0) { s_gmax = 0ULL; s_gmax32 = 0u; s_first = 0x7fffffff; }
        cluster.sync();
        // the other blocks' slices
        for (int g = 0; g < nF; ++g) {
            if (g == f) continue;
            const long long* rw = cluster.map_shared_rank(wq, g);
            const long long* rs = cluster.map_shared_rank(sq, g);
            const int glo = g * ns, ghi = min(J, glo + ns);
            for (int i = glo + tid; i < ghi; i += blockDim.x) {
                wq[i] = rw[i];
                sq[i] = rs[i];
            }
        }
        __syncthreads();
        // prefix sums over this feature's sorted order
        long long pw = 0, ps = 0;
        for (int r = lo; r < hi; ++r) {
            const int k = six[r];
            pw += wq[k];
            ps += sq[k];
        }
        long long pw0 = pw, ps0 = ps, W = 0, S = 0;
        block_scan2(pw0, ps0, red_a, red_b, W, S);
        auto gain = [&](long long WL, long long SL) -> double {
            const long long WR = W - WL, SR = S - SL;
            return (double)SL * (double)SL / (double)WL + (double)SR * (double)SR / (double)WR;
        };
        // The same gain in FP32 (relative error below 4e-7: four conversions, two squares, two
        // divisions and an add, each correctly rounded), used as a filter: a split whose FP32
        // gain is below (1 - 8e-6) times the block's largest FP32 gain is at least 1e-12 below
        // the block's largest exact gain, hence below the tolerance of the overall largest, so
        // the exact FP64 gain is taken only for the splits that pass (the choice is unchanged).
        auto gain32 = [&](long long WL, long long SL) -> float {
            const float a = (float)WL, b = (float)SL, ra = (float)(W - WL), sb = (float)(S - SL);
            return b * b / a + sb * sb / ra;
        };
        {
            float my32 = 0.0f;
            long long a = pw0, b = ps0;
            for (int r = lo; r < hi; ++r) {
                const int k = six[r];
                a += wq[k];
                b += sq[k];
                if (split[r] && a > 0 && W - a > 0) my32 = fmaxf(my32, gain32(a, b));
            }
            atomicMax(&s_gmax32, __float_as_uint(my32));   // gains are >= 0: bits order as values
        }
        __syncthreads();
        const float flt = __uint_as_float(s_gmax32) * (1.0f - 8e-6f);
        unsigned long long my = 0ULL;
        {
            long long a = pw0, b = ps0;
            for (int r = lo; r < hi; ++r) {
                const int k = six[r];
                a += wq[k];
                b += sq[k];
                if (split[r] && a > 0 && W - a > 0 && gain32(a, b) >= flt) {
                    const unsigned long long gb = (unsigned long long)__double_as_longlong(gain(a, b));
                    my = gb > my ? gb : my;
                }
            }
        }
        atomicMax(&s_gmax, my);
        __syncthreads();
        if (tid == 0) {
            lead->gmax[f] = s_gmax;
            if (f == 0) { ex.W = W; ex.S = S; }
        }
        cluster.sync();
        // the overall largest gain (no split included), then this feature's first split within
        // the tolerance; thread 0 reads the leader's values for the block
        if (tid == 0) {
            const long long Wl = lead->W, Sl = lead->S;
            double G = Wl > 0 ? (double)Sl * (double)Sl / (double)Wl : 0.0;
            for (int g = 0; g < nF; ++g) G = fmax(G, __longlong_as_double((long long)lead->gmax[g]));
            s_lim = G * (1.0 - 1e-12);
            s_const = (Wl > 0 && (double)Sl * (double)Sl / (double)Wl >= s_lim) ? 1 : 0;
            s_stop = Wl > 0 ? 0 : 1;          // every weight rounded to 0: nothing to fit
        }
        __syncthreads();
        if (s_stop) break;
        const double lim = s_lim;
        int rfirst = 0x7fffffff;
        long long a_at = 0, b_at = 0;
        if (!s_const) {
            long long a = pw0, b = ps0;
            for (int r = lo; r < hi && rfirst == 0x7fffffff; ++r) {
                const int k = six[r];
                a += wq[k];
                b += sq[k];
                if (split[r] && a > 0 && W - a > 0 && gain32(a, b) >= flt && gain(a, b) >= lim) {
                    rfirst = r;
                    a_at = a;
                    b_at = b;
                }
            }
            atomicMin(&s_first, rfirst);
        }
        __syncthreads();
        const int rstar = s_const ? 0x7fffffff : s_first;
        if (rfirst != 0x7fffffff && rfirst == rstar) {
            lead->cand[f] = rstar;
            lead->cthr[f] = 0.5 * (sv[rstar] + sv[rstar + 1]);
            lead->ccl[f] = (double)b_at / (double)a_at;
            lead->ccr[f] = (double)(S - b_at) / (double)(W - a_at);
        } else if (tid == 0 && rstar == 0x7fffffff) {
            lead->cand[f] = -1;
        }
        for (int wd = warp; wd < nwords; wd += nwarps) {
            const int i = wd * 32 + lane;
            const bool above = i < J && rstar != 0x7fffffff && inv[i] > rstar;
            const unsigned bits = __ballot_sync(FULL, above);
            if (lane == 0) mask[wd] = bits;
        }
        cluster.sync();
        // the chosen stump (thread 0 reads the leader's values) and the update of F's slice
        if (tid == 0) {
            const long long Wl = lead->W, Sl = lead->S;
            int cf = -1;
            if (!s_const)
                for (int g = 0; g < nF && cf < 0; ++g)
                    if (lead->cand[g] >= 0) cf = g;
            if (cf < 0) {
                const double c = Wl > 0 ? (double)Sl / (double)Wl : 0.0;
                s_f = 0; s_thr = -INFINITY; s_cl = c; s_cr = c;
            } else {
                s_f = cf; s_thr = lead->cthr[cf]; s_cl = lead->ccl[cf]; s_cr = lead->ccr[cf];
            }
            if (f == 0) {
                const double B = 0.25 * (s_cr - s_cl), A = 0.25 * (s_cl + s_cr);
                feat[o_st + count] = s_f;
                thr[o_st + count] = s_thr;
                pol[o_st + count] = B >= 0 ? 1 : -1;
                alpha[o_st + count] = fabs(B);
                feat[o_st + count + 1] = s_f;
                thr[o_st + count + 1] = -INFINITY;
                pol[o_st + count + 1] = A >= 0 ? 1 : -1;
                alpha[o_st + count + 1] = fabs(A);
            }
        }
        __syncthreads();
        count += 2;
        {
            const double cl = s_cl, cr = s_cr;
            const bool split_stump = !isinf(s_thr);
            const unsigned* owner = cluster.map_shared_rank(mask, s_f);
            for (int i = s_lo + tid; i < s_hi; i += blockDim.x) {
                const bool above = split_stump ? ((owner[i >> 5] >> (i & 31)) & 1u) != 0 : true;
                Fs[i - s_lo] += 0.5 * (above ? cr : cl);
            }
        }
    }
    if (f == 0 && tid == 0) {
        n_stumps[m] = count;
        stage_cmc_one(nF, count, feat + o_st, thr + o_st, pol + o_st, alpha + o_st, rec_len,
                      rec_f + (size_t)m * rec_len, rec_d + (size_t)m * rec_len);
        fitted[m] = 1;
    }
    cluster.sync();           // the leader's exchange area and the masks stay until all are done
}

// ---------------------------------------------------------------------------------------------
// End of one Newton pass in a graph whose loop is a conditional while node: advance the pass
// index, and continue only while points remain and fewer than max_iter passes ran (each pass has
// its own count and unit counter, zeroed at the date's set-up).

__global__ void newton_decide_kernel(IterState* s, const int* count, int max_iter,
                                     cudaGraphConditionalHandle h, int* passes) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *passes += 1;
    const int it = s->iter;
    const int next_n = count[it + 1];
    s->iter = it + 1;
    cudaGraphSetConditional(h, (next_n > 0 && it + 1 < max_iter) ? 1u : 0u);
}

// ---------------------------------------------------------------------------------------------
// Small helpers.

__global__ void set_int_kernel(int* p, int v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

__global__ void rng_debug_kernel(RoundKeys rk, uint32_t w1, uint32_t step, int d, long long count,
                                 uint32_t* words, double* z) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= count) return;
    const int nc = (d + 3) / 4;
    for (int c = 0; c < nc; ++c) {
        const uint4 x = philox((uint32_t)n, w1, 4u * step + (uint32_t)c, 0u, rk);
        if (words) {
            uint32_t* wo = words + ((size_t)n * nc + c) * 4;
            wo[0] = x.x; wo[1] = x.y; wo[2] = x.z; wo[3] = x.w;
        }
        if (z) {
            float a0, a1;
            PathMath<float>::box_muller(x.x, x.y, a0, a1);
            if (4 * c < d) z[(size_t)n * d + 4 * c] = a0;
            if (4 * c + 1 < d) z[(size_t)n * d + 4 * c + 1] = a1;
            PathMath<float>::box_muller(x.z, x.w, a0, a1);
            if (4 * c + 2 < d) z[(size_t)n * d + 4 * c + 2] = a0;
            if (4 * c + 3 < d) z[(size_t)n * d + 4 * c + 3] = a1;
        }
    }
}

// Counts of items by status (for n_noconv / n_noroot) and the per-date diagnostics copy.
__global__ void collect_points_kernel(const ItemState* state, int n, double* x_out, int* it_out,
                                      int* st_out, int* counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ItemState s = state[i];
    x_out[i] = s.x;
    it_out[i] = s.iters;
    st_out[i] = s.status;
    if (s.status == ST_NOCONV) atomicAdd(&counts[0], 1);
    if (s.status == ST_NOROOT) atomicAdd(&counts[1], 1);
}

__global__ void collect_labels_kernel(const double* label_y, int n, double* x_out, int* it_out,
                                      int* st_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x_out[i] = label_y[i];
    it_out[i] = 1;
    st_out[i] = 0;
}

}  // namespace bap
