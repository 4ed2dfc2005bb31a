// bap_path.cuh -- the nested Monte Carlo path kernel (the hot path).
//
// One launch evaluates continuation sums for a list of items (I&Z boundary points or their
// Newton iterates, CMC training points, or the single pricing start point): Section 2.2 finds
// each boundary point from N_1 simulated paths, Section 3.2 values each training point by
// N_2 further paths started from it.
//
// Work decomposition: an item's N paths are cut into chunks of `chunk` paths (Newton passes left
// with few items: of `tail_chunk` paths); an (item, chunk) unit belongs to one warp, taken from
// a device counter (persistent grid).  Inside a warp every lane runs one path at a time and
// takes the next path index of the chunk as soon as its path stops (warp ballot), so
// early-stopped paths leave no idle lanes.  Results per unit are summed per lane (FP32, flushed
// to FP64 after every block of at most 32 warp steps), reduced across the warp in a fixed
// shuffle tree and written to a fixed slot (the item's position in the pass's list times the
// units per item, plus the unit); the warp that completes an item's last unit sums the slots in
// fixed order, so results are bitwise reproducible whatever the scheduling.  That warp then
// runs the item's epilogue on the device: the Newton update of an I&Z boundary point (and its
// re-queueing), the CMC label, or the plain sums.
#pragma once

#include "bap_internal.cuh"

namespace bap {

struct PathArgs {
    const DevModel* model;
    int m;                       // paths start at t_m and run over t_{m+1}..t_NT
    int mode;                    // Mode
    int n_dates, payoff, uniform;
    double r, K;
    float Lf[MAXD * (MAXD + 1) / 2];   // packed lower Cholesky factor, row q at q(q+1)/2,
                                       // vol-scaled for uniform dates (FP32 kernels)
    float driftf[MAXD];          // uniform dates: per-step log2 drift (FP32 kernels)
    float wf[MAXD];              // basket / geometric weights
    RoundKeys rk;
    int64_t N;                   // paths per item
    int chunk;                   // paths per unit (multiple of 32)
    int C;                       // units per item
    // Newton passes with few items (count * C < tail_units) cut each item into C_tail units of
    // tail_chunk paths instead, so that the few items still spread over the device (0: never).
    // The choice depends on the pass's item count alone, so every launch form makes it alike.
    int tail_chunk, C_tail;
    long long tail_units;
    // Item lists of the passes.  Pass `it` works on the count[it] items list[it & 1][0..) (items
    // 0, 1, ... when that list is null), taking units from the counter work[it]; the Newton
    // epilogue appends the items that go on to list[(it + 1) & 1] at count[it + 1].  Counts and
    // counters are zero before their pass.  `it` is pass_it, or *iter_ptr when iter_ptr is set
    // (graph form), or the pass loop index of the cooperative kernel.
    int* list[2];
    int* count;
    unsigned long long* work;
    int pass_it;
    const int* iter_ptr;
    double* start;               // items x d start points (FP64); Newton writes the pivot value
    float* l0f;                  // items x d: (float) log2 of the start points, kept with them by
                                 // the Newton loop (FP32 kernels; nullptr: taken from start)
    const int* ctr_item;         // Philox counter word 1 per item (nullptr: 0)
    const int* pivot;            // pivot asset per item for the pathwise derivative (or nullptr)
    double* partial;             // per unit 3 sums, at (position in the pass's list) x units
                                 // per item + unit
    long long* partial_steps;    // per unit path-steps, same slots
    int* done;                   // per item: units finished in the current pass
    unsigned long long* total_steps;
    // rule
    int rule_kind;
    const void* rule_src;        // staged rule table (Real), dates 0..n_dates
    int rule_stride;             // Reals per date
    int rules_global;            // read the rows of dates m+1.. from rule_src (a table too large
                                 // for shared memory)
    int row_stride;              // Reals per staged row (set by launch_path: path_row_stride)
    int n_bnd, n_coef, degree;
    const int* fitted;           // n_dates + 1
    // epilogues
    double* out_sums;            // MODE_SUMS / MODE_TRACE: items x 3
    long long* out_steps;
    int* trace_tau;              // MODE_TRACE: per path
    double* trace_phi;
    ItemState* state;            // MODE_NEWTON
    // cooperative Newton loop (newton_coop_kernel): passes run are added to *passes; the grid
    // barrier counts on *coop_bar and flags a timed-out wait in *coop_err
    int* passes;
    unsigned* coop_bar;
    int* coop_err;
    unsigned long long coop_limit_ns;
    double f_tol, x_tol, fp_eps;
    int max_iter, fixed_point;
    int n_items;                 // items the buffers hold (list capacity; bounds checks)
    unsigned long long* checks;  // bounds-check counters of the checked build (or nullptr)
    double* label_y;             // MODE_LABEL: Phi - C
    int* label;                  // +1 exercise / -1 continue
};

// ---------------------------------------------------------------------------------------------
// FP64 payoff at a start point (the item's own point in device memory; used by the Newton and
// label epilogues).  The point is read through L2: in the cooperative Newton loop another SM may
// have moved it in an earlier pass of the same launch.

__device__ inline double payoff64(const PathArgs& a, const double* S, int d) {
    if (a.payoff == BAP_MAX_CALL) {
        double mx = __ldcg(S);
        for (int q = 1; q < d; ++q) mx = fmax(mx, __ldcg(S + q));
        double v = mx - a.K;
        return v > 0 ? v : 0;
    } else if (a.payoff == BAP_BASKET_PUT) {
        double b = 0;
        for (int q = 0; q < d; ++q) b += a.model->w[q] * __ldcg(S + q);
        double v = a.K - b;
        return v > 0 ? v : 0;
    }
    double lg = 0;
    for (int q = 0; q < d; ++q) lg += a.model->w[q] * log(__ldcg(S + q));
    double v = exp(lg) - a.K;
    return v > 0 ? v : 0;
}

// dPhi/dS_p * S_p at S (zero out of the money).
__device__ inline double payoff_dlog64(const PathArgs& a, const double* S, int d, int p) {
    double phi = payoff64(a, S, d);
    if (phi <= 0) return 0;
    if (a.payoff == BAP_MAX_CALL) {
        int best = 0;
        double sb = __ldcg(S);
        for (int q = 1; q < d; ++q) {
            const double sq = __ldcg(S + q);
            if (sq > sb) { sb = sq; best = q; }
        }
        return best == p ? sb : 0.0;
    }
    if (a.payoff == BAP_BASKET_PUT) return -a.model->w[p] * __ldcg(S + p);
    return a.model->w[p] * (phi + a.K);
}

__device__ inline ItemState load_state_l2(const ItemState* p) {
    ItemState s;
    s.x = __ldcg(&p->x);
    s.lo = __ldcg(&p->lo);
    s.hi = __ldcg(&p->hi);
    s.dx_old = __ldcg(&p->dx_old);
    s.dx = __ldcg(&p->dx);
    s.iters = __ldcg(&p->iters);
    s.status = __ldcg(&p->status);
    s.done = __ldcg(&p->done);
    s.pivot = __ldcg(&p->pivot);
    return s;
}

// Newton update of one boundary point after an evaluation of C(x) and C'(x) (FP64; the same
// safeguarded iteration as the reference description: bracket from the signs seen, Newton step
// unless it leaves the bracket or fails to halve the step before last, else bisection, or
// doubling while no upper end is known).  Returns true if the item needs another evaluation.
__device__ inline bool newton_update(const PathArgs& a, int item, double C, double dC) {
    const int d = a.model->d;
    // The item's state and point may have been written on another SM in an earlier pass of
    // the same launch (cooperative form): read them through L2, not a possibly stale L1 line.
    ItemState s = load_state_l2(a.state + item);
    double* S = a.start + (size_t)item * d;
    const int p = s.pivot;
    const double K = a.K;
    double x = s.x;
    s.iters += 1;
    const double phi = payoff64(a, S, d);
    const double f = phi - C;
    const bool put_like = a.payoff == BAP_BASKET_PUT;
    bool done = false;
    double xn = x;
    if (a.fixed_point) {
        if (a.payoff == BAP_MAX_CALL) {
            xn = K + C;
        } else if (a.payoff == BAP_GEO_CALL) {
            double lg = log(K + C);
            for (int q = 0; q < d; ++q)
                if (q != p) lg -= a.model->w[q] * log(__ldcg(S + q));
            xn = exp(lg / a.model->w[p]);
        } else {
            double v = K - C;
            for (int q = 0; q < d; ++q)
                if (q != p) v -= a.model->w[q] * __ldcg(S + q);
            xn = v / a.model->w[p];
            if (xn < 0) xn = 0;
        }
        if (fabs(xn - x) < a.fp_eps) done = true;
        x = xn;
    } else if (fabs(f) < a.f_tol) {
        done = true;
    } else {
        const double dphi = payoff_dlog64(a, S, d, p) / x;
        const double fp = dphi - dC;
        const double sg = put_like ? -1.0 : 1.0;
        const double g = sg * f, gp = sg * fp;
        if (g < 0) s.lo = x; else s.hi = x;
        const double tol = a.x_tol * (fabs(x) > 1.0 ? fabs(x) : 1.0);
        if (s.hi - s.lo <= tol) {
            done = true;
        } else {
            xn = x - g / gp;
            const bool ok = gp > 0 && xn > s.lo && xn < s.hi && fabs(2.0 * g) <= fabs(s.dx_old * gp);
            if (!ok) xn = isinf(s.hi) ? 2.0 * x : 0.5 * (s.lo + s.hi);
            s.dx_old = s.dx;
            s.dx = xn - x;
            if (xn > 1e3 * K) {
                x = 1e3 * K;
                s.status = ST_NOROOT;
                done = true;
            } else if (xn < 1e-6 * K) {
                x = 0.0;
                s.status = ST_NOROOT;
                done = true;
            } else if (fabs(s.dx) <= tol) {
                x = xn;
                done = true;
            } else {
                x = xn;
            }
        }
    }
    if (!done && s.iters >= a.max_iter) {
        s.status = ST_NOCONV;
        done = true;
    }
    s.x = x;
    S[p] = x;
    if (a.l0f) a.l0f[(size_t)item * d + p] = (float)log2(x);
    s.done = done ? 1 : 0;
    a.state[item] = s;
    return !done;
}

// ---------------------------------------------------------------------------------------------

// Resident 256-thread blocks per SM the register budget is sized for (no spills at these),
// with PPL path slots per lane.
template <int D, typename Real, int PPL> constexpr int path_min_blocks() {
    return sizeof(Real) == 8 ? 2 : (PPL > 1 ? (D <= 5 ? 3 : 2) : (D <= 5 ? 4 : (D <= 9 ? 3 : 2)));
}

// Staged rule rows of a launch from date m: dates m+1..NT-1, plus (quadratic I&Z and CMC
// kernels, which evaluate the rule on every step without a per-lane branch) the row of
// maturity, whose result is never used.
__host__ __device__ inline int staged_rule_rows(int rule, int nk) {
    return (rule == R_IZ || rule == R_NEWTON_COOP || rule == R_CMC) ? nk : nk - 1;
}

// Reals per row of the rule rows a kernel reads: a staged CMC row holds the record without its
// overflow area; every other row, and any row read from global memory, is the whole record.
inline int path_row_stride(const PathArgs& a, int rule, int d) {
    return (rule == R_CMC && !a.rules_global) ? cmc_staged_len(d + 1) : a.rule_stride;
}

// Dynamic shared memory of one launch: the staged rule rows first (16-byte aligned), then the
// discount factors, the per-date stepping constants (non-uniform dates only) and the per-date
// "fitted" flags.
inline size_t path_smem_bytes(const PathArgs& a, int rule, bool fp64, int d) {
    const size_t nk = (size_t)(a.n_dates - a.m);
    const size_t row = (size_t)path_row_stride(a, rule, d);
    const size_t n = (rule != R_NONE && !a.rules_global
                          ? (size_t)staged_rule_rows(rule, (int)nk) * row : 0) +
                     nk + (a.uniform ? 0 : 2 * nk * (size_t)d);
    return n * (fp64 ? 8 : 4) + nk * sizeof(int);
}

// The stump rule F(S) of a record in which some feature keeps its thresholds in the overflow
// area (bit f of ovf), read from the record in global memory: the same sum in the same order,
// each count taken by a plain binary search (a rare path: features with 32 or more distinct
// thresholds).  An overflow entry that does not fit the record counts nothing.
template <int NF, int D, typename Real>
__device__ __forceinline__ Real cmc_rule_overflow(const Real* rec, int ovf, int stride,
                                                  const Real (&S)[D], Real phi) {
    Real F = rec[0];
#pragma unroll 1
    for (int f = 0; f < NF; ++f) {
        Real xv = phi;
#pragma unroll
        for (int q = 0; q < D; ++q) xv = (f == q) ? S[q] : xv;
        const Real* blk = rec + CMC_HEAD + 2 * CMC_SLOTS * f;
        const Real* t = blk;
        int n = CMC_SLOTS;
        if ((ovf >> f) & 1) {
            const int off = get_int_as(blk[0]);
            n = get_int_as(blk[1]);
            const int base = CMC_HEAD + 2 * CMC_SLOTS * NF;
            if (n < 0 || n > BAP_MAX_STUMPS || off < base || off > stride - 2 * n - 1) continue;
            t = rec + off;
        }
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (t[mid] < xv) lo = mid + 1; else hi = mid;
        }
        F += t[(t == blk ? CMC_SLOTS : n) + lo];
    }
    return F;
}

// Loads N consecutive values from 16-byte-aligned shared memory with vector loads.
template <int N>
__device__ __forceinline__ void load_vec(const float* src, float (&dst)[N]) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
        const float4 v = s4[i];
        dst[4 * i] = v.x; dst[4 * i + 1] = v.y; dst[4 * i + 2] = v.z; dst[4 * i + 3] = v.w;
    }
}
template <int N>
__device__ __forceinline__ void load_vec(const double* src, double (&dst)[N]) {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const double2 v = s2[i];
        dst[2 * i] = v.x; dst[2 * i + 1] = v.y;
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned load_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch with a bounded wait.  *bar counts block arrivals
// over the whole launch (zero before it); a barrier is passed once the count reaches `target`,
// the arrivals of all barriers so far (the blocks still running at each).  A block that waits
// longer than limit_ns, or sees *err set by another block, sets *err and gets false: the caller
// then leaves the kernel, so every block ends in bounded time and the host reads the flag.
__device__ inline bool grid_barrier(unsigned* bar, unsigned target, int* err, unsigned long long limit_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned long long t0 = global_ns();
        while (load_acquire_gpu(bar) < target) {
            if (*(volatile int*)err != 0 || global_ns() - t0 > limit_ns) {
                atomicExch(err, 1);
                good = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// The path kernel.  PAY >= 0 specialises it for one payoff (the FP32 quadratic I&Z kernels);
// -1 reads the payoff from the arguments.  Plain form (COOP = false): one pass, `it` = pass_it
// or *iter_ptr.
// Cooperative form (COOP = true, I&Z Newton only): every Newton pass of one date in one launch,
// it = 0, 1, ..., on the same lists, counts and unit counters as the plain form (all zero
// before the launch); a grid barrier ends each pass, after which all blocks read the same next
// count, so all run the same passes.  Its grid must be co-resident (cudaLaunchCooperativeKernel
// checks that); the barrier's wait is bounded all the same (coop_err, coop_limit_ns).
// The unit loop is written once, in this kernel body: moved into an inlined device function it
// compiled measurably slower.
template <int D, int RULE, typename Real, bool COOP, int PPL = 1, int PAY = -1>
__global__ void __launch_bounds__(256, (path_min_blocks<D, Real, PPL>())) path_kernel(const PathArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // each thread's FP64 partial sums of its unit (kept here rather than in six registers)
    __shared__ double sh_sum[3][256];
    constexpr int NF = D + 1;
    constexpr int P4 = (RULE == R_IZ3) ? iz_stage_stride3(D) : iz_stage_stride(D);
    const int nk = a.n_dates - a.m;                  // dates m+1..NT
    // rows of dates m+1..NT-1, staged in shared memory (read from global memory for a table
    // too large to stage); a CMC row is staged without its overflow area, at an odd row length
    const bool rules_global = a.rules_global != 0;
    const int row_stride = a.row_stride;
    const int rule_len = (RULE == R_NONE || rules_global) ? 0 : staged_rule_rows(RULE, nk) * row_stride;
    Real* sh_rule = reinterpret_cast<Real*>(smem_raw);
    Real* sh_disc = sh_rule + rule_len;
    Real* sh_drift = sh_disc + nk;                   // non-uniform dates: [nk][D]
    Real* sh_vol = sh_drift + (a.uniform ? 0 : nk * D);
    int* sh_fit = reinterpret_cast<int*>(sh_vol + (a.uniform ? 0 : nk * D));

    const DevModel* M = a.model;
    const Real* rule_rows = sh_rule;
    // the global rows of dates m+1.. (a CMC record's overflow area is read there)
    const Real* rule_src = RULE == R_NONE ? nullptr
        : reinterpret_cast<const Real*>(a.rule_src) + (size_t)(a.m + 1) * a.rule_stride;
    if (RULE != R_NONE) {
        if (RULE == R_CMC && !rules_global) {
            constexpr int FIXED = CMC_HEAD + 2 * CMC_SLOTS * NF;
            const int rows = staged_rule_rows(RULE, nk);
            for (int r = 0; r < rows; ++r)
                for (int c = threadIdx.x; c < row_stride; c += blockDim.x)
                    sh_rule[r * row_stride + c] = c < FIXED ? rule_src[(size_t)r * a.rule_stride + c] : (Real)0;
        } else {
            for (int i = threadIdx.x; i < rule_len; i += blockDim.x) sh_rule[i] = rule_src[i];
        }
        if (rules_global) rule_rows = rule_src;
    }
    for (int i = threadIdx.x; i < nk; i += blockDim.x) {
        const int k = a.m + 1 + i;
        sh_disc[i] = (Real)exp(-a.r * (M->t[k] - M->t[a.m]));
        sh_fit[i] = (a.fitted != nullptr && k < a.n_dates) ? a.fitted[k] : 0;
    }
    if (!a.uniform) {
        for (int i = threadIdx.x; i < nk * D; i += blockDim.x) {
            const int k = a.m + 1 + i / D, q = i % D;
            sh_drift[i] = (Real)M->drift2[k][q];
            sh_vol[i] = (Real)M->vol2[k][q];
        }
    }
    __syncthreads();

    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    const Real K = (Real)a.K;
    // the payoff: a template constant in the specialised kernels (PAY >= 0), else the argument's
    const int payoff = PAY >= 0 ? PAY : a.payoff;
    const bool is_put = payoff == BAP_BASKET_PUT;
    const bool is_max = payoff == BAP_MAX_CALL;

    // The Cholesky factor and the per-step drift are read straight from the kernel parameters
    // (constant bank operands, no registers).
    // (The FP64 check kernels read them from the device model instead.)
    auto Lc = [&](int q, int j) -> Real {
        if constexpr (sizeof(Real) == 4) return a.Lf[q * (q + 1) / 2 + j];
        else return M->L[q * MAXD + j] * (a.uniform ? M->vol2[1][q] : 1.0);
    };
    auto drift_c = [&](int q) -> Real {
        if constexpr (sizeof(Real) == 4) return a.driftf[q];
        else return M->drift2[1][q];
    };


    int it = COOP ? 0 : (a.iter_ptr ? *a.iter_ptr : a.pass_it);
    bool ok = true;
    // cooperative form: the blocks that run the current pass (0 .. active-1), and the barrier
    // count that ends it
    unsigned active = gridDim.x, bar_target = 0;
    for (;;) {
    // ---- one pass: every unit of the count[it] items of list[it & 1] ----
    const int pass_count = __ldcg(a.count + it);
    int pass_chunk = a.chunk, pass_C = a.C;
    if (a.tail_chunk > 0 && (long long)pass_count * a.C < a.tail_units) {
        pass_chunk = a.tail_chunk;
        pass_C = a.C_tail;
    }
    const long long total_units = (long long)pass_count * pass_C;
        while (true) {
            unsigned long long unit_u = 0;
            if (lane == 0) unit_u = atomicAdd(a.work + it, 1ULL);
            const long long unit = (long long)__shfl_sync(FULL, unit_u, 0);
            if (unit >= total_units) break;
            const int slot = (int)(unit / pass_C);
            const int chunk = (int)(unit - (long long)slot * pass_C);
            // the unit's partial-sum slot, slot * pass_C + chunk = unit (fewer than 2^32 slots;
            // the launcher checks): kept instead of slot and chunk, which the epilogue re-derives
            const unsigned unit_o = (unsigned)unit;
            const int* active = a.list[it & 1];
            const int item = active ? __ldcg(active + slot) : slot;
            if (!bap_check(item >= 0 && item < a.n_items, 1, a.checks)) continue;

            // log2 of the start point, one coordinate per lane, then broadcast: kept per item by
            // the Newton loop (the same FP64 log2 rounded to FP32), else taken here in FP64
            Real l0[D];
            if (sizeof(Real) == 4 && a.l0f != nullptr) {
                const float my_l0 = lane < D ? __ldcg(a.l0f + (size_t)item * D + lane) : 0.f;
#pragma unroll
                for (int q = 0; q < D; ++q) l0[q] = (Real)__shfl_sync(FULL, my_l0, q);
            } else {
                const double* st = a.start + (size_t)item * D;
                const double my_l0 = lane < D ? log2(__ldcg(st + lane)) : 0.0;
#pragma unroll
                for (int q = 0; q < D; ++q) l0[q] = (Real)__shfl_sync(FULL, my_l0, q);
            }
            const int pivot = a.pivot ? a.pivot[item] : -1;
            // The unit covers paths n_begin .. n_begin + n_count - 1.  Inside the loop only the
            // 32-bit offset nl moves: counter word 0 is (n_begin + nl) mod 2^32 and word 1 stays
            // item + n_begin / 2^32 (a unit never straddles a multiple of 2^32 paths).
            const long long n_begin = (long long)chunk * pass_chunk;
            const int n_count = (int)min((long long)pass_chunk, (long long)a.N - n_begin);
            const uint32_t w0_base = (uint32_t)n_begin;
            const uint32_t w1_word = (a.ctr_item ? (uint32_t)a.ctr_item[item] : 0u) + (uint32_t)(n_begin >> 32);

            // PPL path slots per lane: slot s of lane L starts with path s * 32 + L; a slot whose
            // path stops takes the next path index of the unit (slot-major order across the warp,
            // by ballot), so early-stopped paths leave no idle slots.  Several slots give the
            // scheduler independent instruction streams within one warp.
            int nl[PPL], k[PPL];
            bool has[PPL];
            Real l[PPL][D];
#pragma unroll
            for (int s = 0; s < PPL; ++s) {
                nl[s] = s * 32 + lane;
                has[s] = nl[s] < n_count;
                k[s] = a.m;
#pragma unroll
                for (int q = 0; q < D; ++q) l[s][q] = l0[q];
            }
            int next = 32 * PPL;
            Real acc0 = 0, acc1 = 0, acc2 = 0;
            sh_sum[0][threadIdx.x] = 0.0;
            sh_sum[1][threadIdx.x] = 0.0;
            sh_sum[2][threadIdx.x] = 0.0;
            int steps = 0;

            // Blocks of up to 32 warp steps; the FP32 partial sums move to FP64 after each block
            // (a lane ends at most 32 PPL paths in between).  The flush sits outside the inner loop
            // on purpose: inside it the compiler would evaluate it speculatively on every step, and
            // the FP64 pipe runs at 1/64 of the FP32 rate.
            bool live = true;
            while (live) {
            for (int it = 0; it < 32; ++it) {
                bool any_has = false;
#pragma unroll
                for (int s = 0; s < PPL; ++s) any_has = any_has || has[s];
                live = __any_sync(FULL, any_has);
                if (!live) break;
                bool finished[PPL];
                // The step of every slot, without a branch: a slot with no path left steps a
                // throw-away path from date m (so that every index stays in range) and none of
                // its results count.
#pragma unroll
                for (int s = 0; s < PPL; ++s) {
                    k[s] = has[s] ? k[s] + 1 : a.m + 1;
                    steps += has[s] ? 1 : 0;
                    const int ks = k[s];
                    Real z[D];
                    normals<D, Real>(w0_base + (uint32_t)nl[s], w1_word, (uint32_t)ks, a.rk, z);
                    if (a.uniform) {
                        // l_q += drift_q + sum_j L'_qj z_j (L' the vol-scaled factor), the drift
                        // taken as the first term of the sum
#pragma unroll
                        for (int q = 0; q < D; ++q) {
                            Real wq = drift_c(q);
#pragma unroll
                            for (int j = 0; j <= q; ++j) wq = fma(Lc(q, j), z[j], wq);
                            l[s][q] = l[s][q] + wq;
                        }
                    } else {
                        const int kk = (ks - a.m - 1) * D;
#pragma unroll
                        for (int q = 0; q < D; ++q) {
                            Real wq = 0;
#pragma unroll
                            for (int j = 0; j <= q; ++j) wq = fma(Lc(q, j), z[j], wq);
                            l[s][q] = fma(sh_vol[kk + q], wq, l[s][q] + sh_drift[kk + q]);
                        }
                    }
                    // prices and payoff
                    Real S[D];
#pragma unroll
                    for (int q = 0; q < D; ++q) S[q] = PathMath<Real>::exp2r(l[s][q]);
                    int imax = 0;
                    Real lmax = l[s][0];
#pragma unroll
                    for (int q = 1; q < D; ++q)
                        if (l[s][q] > lmax) { lmax = l[s][q]; imax = q; }
                    Real phi;
                    Real gval = 0;
                    Real sp;                 // the price tested against the boundary
                    if (is_max) {
                        sp = PathMath<Real>::exp2r(lmax);      // = S[imax], the same operation
                        phi = sp - K;
                    } else if (is_put) {
                        Real b = 0;
#pragma unroll
                        for (int q = 0; q < D; ++q) b = fma((Real)a.wf[q], S[q], b);
                        phi = K - b;
                        sp = S[0];
                    } else {
                        Real lg = 0;
#pragma unroll
                        for (int q = 0; q < D; ++q) lg = fma((Real)a.wf[q], l[s][q], lg);
                        gval = PathMath<Real>::exp2r(lg);
                        phi = gval - K;
                        sp = S[0];
                    }
                    const int kr = ks - a.m - 1;
                    bap_check(kr >= 0 && kr < a.n_dates - a.m, 5, a.checks);
                    const bool at_T = ks == a.n_dates;
                    bool ex = phi > 0;
                    if constexpr (RULE == R_IZ) {
                        // exercise iff S_p passes B_p(S), the pivot p = argmax for the max-call;
                        // evaluated on every step without a branch (the staged table has a zero
                        // row for maturity, where only the payoff decides)
                        Real cc[P4];
                        load_vec<P4>(rule_rows + kr * row_stride + (is_max ? imax : 0) * P4, cc);
                        Real B = cc[0];
                        int idx = 1;
#pragma unroll
                        for (int t = 0; t < D; ++t) {
                            Real acc = cc[idx++];
#pragma unroll
                            for (int u = t; u < D; ++u) acc = fma(cc[idx++], S[u], acc);
                            B = fma(acc, S[t], B);
                        }
                        const bool exr = is_put ? (sp <= B) : (sp >= B);
                        ex = ex && (at_T || (sh_fit[kr] != 0 && exr));
                    } else if constexpr (RULE == R_CMC) {
                        // F(S) = F0 + sum_f T_f[#{t_f < x_f}], for every lane of a warp in which
                        // some lane needs it (a path in the money before maturity)
                        const bool need = ex && !at_T && has[s];
                        if (__any_sync(FULL, need)) {
                            const Real* rec = rule_rows + kr * row_stride;
                            Real F = rec[0];
#pragma unroll
                            for (int f = 0; f < NF; ++f) {
                                const Real xv = f < D ? S[f < D ? f : 0] : phi;
                                // five-level search of the block's CMC_SLOTS sorted values
                                // (+inf padded): p ends at t_f + #{t_f < x}
                                const Real* p = rec + CMC_HEAD + 2 * CMC_SLOTS * f;
#pragma unroll
                                for (int step = CMC_SLOTS / 2; step >= 1; step >>= 1)
                                    p = (p[step - 1] < xv) ? p + step : p;
                                F += p[CMC_SLOTS];
                            }
                            const int ovf = get_int_as(rec[1]);
                            if (ovf != 0) {
                                const Real* rec_g = reinterpret_cast<const Real*>(a.rule_src) +
                                                    (size_t)(a.m + 1 + kr) * a.rule_stride;
                                F = cmc_rule_overflow<NF>(rec_g, ovf, a.rule_stride, S, phi);
                            }
                            ex = ex && (at_T || (sh_fit[kr] != 0 && F > 0));
                        } else {
                            ex = ex && at_T;
                        }
                    } else if (ex && !at_T) {
                        if (RULE == R_NONE || !sh_fit[kr]) {
                            ex = false;
                        } else if (RULE == R_IZ3) {
                            // the cubic boundary in the d-1 other prices (nested Horner order);
                            // the coefficients are read from shared memory as they are used
                            const int p = is_max ? imax : 0;
                            const Real* cc = rule_rows + kr * row_stride + (a.n_bnd > 1 ? p : 0) * P4;
                            Real B = cc[0];
                            if constexpr (D > 1) {
                                Real y[D - 1];
#pragma unroll
                                for (int t = 0; t < D - 1; ++t) y[t] = (t < p) ? S[t] : S[t + 1];
                                int idx = 1;
#pragma unroll
                                for (int t = 0; t < D - 1; ++t) {
                                    Real acc_t = cc[idx++];
#pragma unroll
                                    for (int u = t; u < D - 1; ++u) {
                                        Real acc_u = cc[idx++];
#pragma unroll
                                        for (int v = u; v < D - 1; ++v) acc_u = fma(cc[idx++], y[v], acc_u);
                                        acc_t = fma(acc_u, y[u], acc_t);
                                    }
                                    B = fma(acc_t, y[t], B);
                                }
                            }
                            ex = is_put ? (sp <= B) : (sp >= B);
                        }
                    }
                    ex = ex && has[s];
                    finished[s] = has[s] && (ex || at_T);
                    // discounted payoff of a path that stops here (0 if it is not exercised) and
                    // its pathwise derivative with respect to the pivot's start value
                    const Real disc = sh_disc[kr];
                    const Real v = ex ? disc * phi : (Real)0;
                    Real dv = 0;
                    if (pivot >= 0) {
                        if (is_max) {
                            dv = (imax == pivot) ? disc * (phi + K) : (Real)0;
                        } else if (is_put) {
                            Real spv = S[0], wp = (Real)a.wf[0];
#pragma unroll
                            for (int q = 1; q < D; ++q) {
                                spv = (q == pivot) ? S[q] : spv;
                                wp = (q == pivot) ? (Real)a.wf[q] : wp;
                            }
                            dv = -disc * wp * spv;
                        } else {
                            Real wp = (Real)a.wf[0];
#pragma unroll
                            for (int q = 1; q < D; ++q) wp = (q == pivot) ? (Real)a.wf[q] : wp;
                            dv = disc * wp * gval;
                        }
                        dv = ex ? dv : (Real)0;
                    }
                    if (a.mode == MODE_TRACE && finished[s]) {
                        if (bap_check(n_begin + nl[s] < a.N, 3, a.checks)) {
                            a.trace_tau[n_begin + nl[s]] = ex ? ks : a.n_dates + 1;
                            a.trace_phi[n_begin + nl[s]] = (double)v;
                        }
                    }
                    acc0 += v;
                    acc1 += v * v;
                    acc2 += dv;
                }
                // stopped paths take the next path indices of the unit, slot by slot
#pragma unroll
                for (int s = 0; s < PPL; ++s) {
                    const unsigned need = __ballot_sync(FULL, finished[s]);
                    if (finished[s]) {
                        nl[s] = next + __popc(need & lanemask_lt);
                        has[s] = nl[s] < n_count;
#pragma unroll
                        for (int q = 0; q < D; ++q) l[s][q] = l0[q];
                        k[s] = a.m;
                    }
                    next += __popc(need);
                }
            }
            sh_sum[0][threadIdx.x] += (double)acc0;
            sh_sum[1][threadIdx.x] += (double)acc1;
            sh_sum[2][threadIdx.x] += (double)acc2;
            acc0 = acc1 = acc2 = 0;
            }
            long long steps64 = steps;
            double s0 = sh_sum[0][threadIdx.x], s1 = sh_sum[1][threadIdx.x], s2 = sh_sum[2][threadIdx.x];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                s0 += __shfl_down_sync(FULL, s0, off);
                s1 += __shfl_down_sync(FULL, s1, off);
                s2 += __shfl_down_sync(FULL, s2, off);
                steps64 += __shfl_down_sync(FULL, steps64, off);
            }
            int last = 0;
            if (lane == 0) {
                const size_t o = unit_o;
                a.partial[3 * o + 0] = s0;
                a.partial[3 * o + 1] = s1;
                a.partial[3 * o + 2] = s2;
                a.partial_steps[o] = steps64;
                __threadfence();
                last = atomicAdd(&a.done[item], 1) == pass_C - 1;
            }
            last = __shfl_sync(FULL, last, 0);
            if (!last) continue;

            // ---- the warp that finished the item's last unit: fixed-order sum over its units ----
            __threadfence();
            const int unit_chunk = (int)(n_begin / pass_chunk);
            bap_check(unit_chunk >= 0 && unit_chunk < pass_C, 4, a.checks);
            const size_t o_first = (size_t)unit_o - unit_chunk;    // slot * pass_C
            double t0 = 0, t1 = 0, t2 = 0;
            long long ts = 0;
            for (int c = lane; c < pass_C; c += 32) {
                const size_t o = o_first + c;
                t0 += __ldcg(a.partial + 3 * o + 0);
                t1 += __ldcg(a.partial + 3 * o + 1);
                t2 += __ldcg(a.partial + 3 * o + 2);
                ts += __ldcg(a.partial_steps + o);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                t0 += __shfl_down_sync(FULL, t0, off);
                t1 += __shfl_down_sync(FULL, t1, off);
                t2 += __shfl_down_sync(FULL, t2, off);
                ts += __shfl_down_sync(FULL, ts, off);
            }
            if (lane == 0) {
                a.done[item] = 0;
                atomicAdd(a.total_steps, (unsigned long long)ts);
                const double Nd = (double)a.N;
                if (a.mode == MODE_SUMS || a.mode == MODE_TRACE) {
                    // the pathwise derivative is with respect to the pivot's start value x
                    const int pv = a.pivot ? a.pivot[item] : -1;
                    const double xs = (pv >= 0 && pv < D) ? a.start[(size_t)item * D + pv] : 1.0;
                    a.out_sums[3 * item + 0] = t0;
                    a.out_sums[3 * item + 1] = t1;
                    a.out_sums[3 * item + 2] = t2 / xs;
                    a.out_steps[item] = ts;
                } else if (a.mode == MODE_NEWTON) {
                    const double x = __ldcg(&a.state[item].x);
                    if (newton_update(a, item, t0 / Nd, t2 / (Nd * x))) {
                        const int pos = atomicAdd(a.count + it + 1, 1);
                        if (bap_check(pos >= 0 && pos < a.n_items, 2, a.checks))
                            a.list[(it + 1) & 1][pos] = item;
                    }
                } else if (a.mode == MODE_LABEL) {
                    const double phi = payoff64(a, a.start + (size_t)item * D, D);
                    const double y = phi - t0 / Nd;
                    a.label_y[item] = y;
                    a.label[item] = y > 0 ? 1 : -1;
                }
            }
        }
    if constexpr (!COOP) break;
    bar_target += active;
    ok = grid_barrier(a.coop_bar, bar_target, a.coop_err, a.coop_limit_ns);
    if (!ok) break;
    const int next_count = __ldcg(a.count + it + 1);
    if (next_count == 0 || it + 1 >= a.max_iter) break;
    // blocks beyond what the next pass's units can occupy leave, so that their SMs serve other
    // work (every block reads the same count, so all agree on who stays)
    const int next_C = (a.tail_chunk > 0 && (long long)next_count * a.C < a.tail_units) ? a.C_tail : a.C;
    const long long need = ((long long)next_count * next_C + (blockDim.x / 32) - 1) / (blockDim.x / 32);
    if (need < (long long)active) active = (unsigned)need;
    if (blockIdx.x >= active) break;
    ++it;
    }
    if (COOP && ok && blockIdx.x == 0 && threadIdx.x == 0 && a.passes) *a.passes += it + 1;
}

}  // namespace bap
