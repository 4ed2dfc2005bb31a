// bap_api.cu -- host side of the C ABI declared in include/bap.h.
//
// The host validates arguments, owns device buffers and enqueues kernels on the option's
// stream.  The FP64 Cholesky factorisation of rho (a few hundred flops per option, the
// positive-definiteness check) runs on the host when the option is created; every other step
// of the method (lattice, Newton iterations, regression, training points, boosting, pricing)
// runs in device kernels, and the host reads back only the results a call returns.  Fits and pricing are split into an enqueue part (asynchronous on the
// option's stream, results into page-locked host memory) and a finish part, so that the serving
// loop can keep many options in flight.
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bap_host.cuh"

using namespace bap;

namespace bap {

static thread_local std::string g_err;

bap_status fail(bap_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

void clear_error() { g_err.clear(); }

cudaStream_t& alloc_stream() {
    static thread_local cudaStream_t s = nullptr;
    return s;
}

static std::mutex g_pin_mu;
static std::vector<PinnedOut*> g_pin_free;

PinnedOut* pinned_get() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        const int n = 256;
        PinnedOut* slab = nullptr;
        if (cudaMallocHost(&slab, sizeof(PinnedOut) * n) != cudaSuccess) return nullptr;
        for (int i = n - 1; i >= 0; --i) g_pin_free.push_back(slab + i);
    }
    PinnedOut* p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}

void pinned_put(PinnedOut* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

// Keep freed pool memory cached in the process (a process-local pool attribute), so that the
// stream-ordered allocations of successive options reuse it instead of returning it.
void keep_pool_cached(int dev) {
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long thr = ~0ULL;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

const char* error_text() { return g_err.c_str(); }

}  // namespace bap

namespace {

constexpr int kBlock = 256;

// Per (kernel, device): whether its dynamic shared-memory limit is raised, and the cached
// occupancy for the last shared-memory size asked about.
struct FnInfo {
    bool smem_raised = false;
    size_t max_dyn_smem = 0;          // the raised limit

    size_t occ_smem = ~size_t(0);
    int occ_blocks = 0;
};
std::mutex g_fn_mu;
std::map<std::pair<const void*, int>, FnInfo> g_fn;

// Raise a kernel's dynamic shared-memory limit to everything the device allows, once per device
// (call with g_fn_mu held).  Changing the attribute waits for running launches of the kernel,
// so it must not happen again once requests are in flight.
bap_status raise_smem_limit(const void* fn, int device, FnInfo& fi) {
    if (fi.smem_raised) return BAP_OK;
    int optin = 0;
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    cudaFuncAttributes fa;
    CU(cudaFuncGetAttributes(&fa, fn));
    CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
    fi.max_dyn_smem = (size_t)(optin - (int)fa.sharedSizeBytes);
    fi.smem_raised = true;
    return BAP_OK;
}

// Resident blocks per SM of a path kernel at this dynamic shared-memory size.
bap_status path_blocks_per_sm(const void* fn, int device, size_t smem, int* bps) {
    std::lock_guard<std::mutex> lk(g_fn_mu);
    FnInfo& fi = g_fn[{fn, device}];
    TRY(raise_smem_limit(fn, device, fi));
    if (fi.occ_smem != smem) {
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fi.occ_blocks, fn, kBlock, smem));
        fi.occ_smem = smem;
    }
    *bps = std::max(1, fi.occ_blocks);
    return BAP_OK;
}

const void* path_fn(int D, int rule, bool fp64, int ppl = 1, int payoff = -1) {
    switch (D) {
        case 1: return path_kernel_fn<1>(rule, fp64, ppl, payoff);
        case 2: return path_kernel_fn<2>(rule, fp64, ppl, payoff);
        case 3: return path_kernel_fn<3>(rule, fp64, ppl, payoff);
        case 4: return path_kernel_fn<4>(rule, fp64, ppl, payoff);
        case 5: return path_kernel_fn<5>(rule, fp64, ppl, payoff);
        case 6: return path_kernel_fn<6>(rule, fp64, ppl, payoff);
        case 7: return path_kernel_fn<7>(rule, fp64, ppl, payoff);
        case 8: return path_kernel_fn<8>(rule, fp64, ppl, payoff);
        case 9: return path_kernel_fn<9>(rule, fp64, ppl, payoff);
        case 10: return path_kernel_fn<10>(rule, fp64, ppl, payoff);
        default: return nullptr;
    }
}

bool has_device(int* dev) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return false;
    return cudaGetDevice(dev) == cudaSuccess;
}

// Paths per warp unit: a function of the launch shape (and of the option's unit setting) only,
// so that results do not depend on what else runs.  Automatic (unit_paths = 0): about 16k
// units, 64..2048 paths each, a multiple of 32; else unit_paths (a multiple of 32).
int choose_chunk(long long n_items, long long N, int unit_paths = 0) {
    long long target = (n_items * N + 16383) / 16384;
    long long c = ((target + 31) / 32) * 32;
    c = std::max(64LL, std::min(2048LL, c));
    if (unit_paths > 0) c = unit_paths;
    long long nr = ((N + 31) / 32) * 32;
    c = std::min(c, std::max(32LL, nr));
    // very long pricing runs: keep the unit count below 2^24
    while ((N + c - 1) / c > (1LL << 24)) c *= 2;
    // beyond 2^32 paths the counter's high word must stay fixed inside a unit: a power-of-two
    // unit never straddles a multiple of 2^32
    if (N > (1LL << 32)) {
        long long p2 = 64;
        while (p2 < c) p2 <<= 1;
        c = p2;
    }
    return (int)c;
}

// The unit of the Newton passes with few items: a power of two, at most an eighth of the main
// unit, at least 64 paths (0: main units under 512 paths are not cut).
int tail_chunk_for(int chunk) {
    if (chunk < 512) return 0;
    int t = 64;
    while (t * 2 <= chunk / 8) t *= 2;
    return t;
}

// The tail split of a date's Newton launch over n items: passes whose units number fewer than
// tail_units (two per resident warp of the device, or a quarter of the first pass's) run on
// the smaller units.
long long tail_units_for(long long n, int C, int sm_count) {
    return std::min(2LL * 32 * sm_count, n * C / 4);
}

void set_tail_split(const bap_option* o, PathArgs& a) {
    a.tail_chunk = tail_chunk_for(a.chunk);
    if (a.tail_chunk == 0) return;
    a.C_tail = (int)((a.N + a.tail_chunk - 1) / a.tail_chunk);
    a.tail_units = tail_units_for(o->n_items, a.C, o->sm_count);
}

// Unit-partial slots of the Newton launches over n items (slots are numbered by an item's
// position in its pass's list): n C for a main pass, fewer than tail_units / C items times the
// tail units per item for a tail pass.
long long newton_unit_slots(long long n, long long N, int chunk, int sm_count) {
    const long long C = (N + chunk - 1) / chunk;
    const int t = tail_chunk_for(chunk);
    if (t == 0) return n * C;
    const long long tail_items = std::min(n, tail_units_for(n, (int)C, sm_count) / C + 1);
    return std::max(n * C, tail_items * ((N + t - 1) / t));
}

// ---- launch configuration from the autotuner's table ------------------------------------------
// bap_tuning.inc holds, per launch shape measured on the target GPU by the project's autotuner
// (autotune.py), the fastest paths per warp unit and path slots per lane of the quadratic I&Z
// Newton launches (kind 0) and the paths per warp unit of the CMC label launches (kind 1):
// entries {d, kind, items, N, unit paths, slots per lane}.  A fit takes the entry of its kind
// and d nearest to its shape (log distance in items and paths); without one, the fixed formula
// of choose_chunk and one slot per lane.
struct TuneEntry {
    int d, kind, items;
    long long N;
    int unit, ppl;
};
const TuneEntry kTune[] = {
#include "bap_tuning.inc"
    {0, -1, 0, 0, 0, 0}};

struct LaunchChoice {
    int unit = 0;         // 0: the formula
    int ppl = 1;
    bool tuned = false;
};

LaunchChoice tuned_launch(int d, int kind, long long n_items, long long N) {
    LaunchChoice c;
    double best = 1e300;
    for (const TuneEntry& e : kTune) {
        if (e.kind != kind || e.d != d || e.items <= 0 || e.N <= 0) continue;
        const double dist = std::fabs(std::log((double)n_items / e.items)) +
                            std::fabs(std::log((double)N / (double)e.N));
        if (dist < best) {
            best = dist;
            c.unit = e.unit;
            c.ppl = e.ppl;
            c.tuned = true;
        }
    }
    return c;
}

// The tuning kind of a fit: 0 the quadratic (or lower) I&Z Newton launches, 1 the CMC label
// launches; cubic boundaries (-1) take the formula.  The choice depends on the fit's shape
// only, never on what else runs or on the device share, so a fit's result is the same alone
// and served.
int tune_kind(int method, int degree) {
    if (method == BAP_METHOD_CMC) return 1;
    return degree <= 2 ? 0 : -1;
}

// The kernel for a rule: a cubic I&Z boundary has kernels of its own.
int kernel_rule(const bap_option* o, int rule) {
    if (o->rule_kind == R_IZ && o->degree >= 3) {
        if (rule == R_IZ) return R_IZ3;
        if (rule == R_NEWTON_COOP) return R_NEWTON_COOP3;
    }
    return rule;
}

// no_events: never create profiling events (the allocation-free entry point creates nothing).
bap_status launch_path(bap_option* o, PathArgs& a, int rule, bool fp64, long long max_units,
                       bool no_events = false) {
    rule = kernel_rule(o, rule);
    // path slots per lane: the option's setting, else the tuned choice of the fit's Newton launches
    const int ppl = o->ppl ? o->ppl : (a.mode == MODE_NEWTON ? o->ppl_fit : 1);
    const void* fn = path_fn(o->d, rule, fp64, ppl, o->payoff);
    if (!fn) return fail(BAP_EINVAL, "no path kernel for d=%d", o->d);
    // the dynamic shared memory the kernel may use (the device's limit less its static arrays)
    size_t max_smem = 0;
    {
        std::lock_guard<std::mutex> lk(g_fn_mu);
        FnInfo& fi = g_fn[{fn, o->device}];
        TRY(raise_smem_limit(fn, o->device, fi));
        max_smem = fi.max_dyn_smem;
    }
    size_t smem = path_smem_bytes(a, rule, fp64, o->d);
    if (smem > max_smem && rule != R_NONE) {
        // a table too large to stage (many dates, many coefficients or stumps; the FP64
        // re-runs first): the kernel reads the rule rows from global memory instead
        a.rules_global = 1;
        smem = path_smem_bytes(a, rule, fp64, o->d);
    }
    a.row_stride = path_row_stride(a, rule, o->d);
    if (smem > max_smem) return fail(BAP_EINVAL, "rule tables too large for shared memory (%zu B)", smem);
    int bps = 1;
    TRY(path_blocks_per_sm(fn, o->device, smem, &bps));
    long long blocks = (max_units + (kBlock / 32) - 1) / (kBlock / 32);
    long long cap = (long long)o->sm_count * bps;
    const bool coop = rule == R_NEWTON_COOP || rule == R_NEWTON_COOP3;
    if (coop) cap = std::max(1LL, cap / std::max(1, o->grid_share));
    blocks = std::max(1LL, std::min(blocks, cap));
    void* args[] = {&a};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = o->profiling && !fp64 && !o->capturing && !no_events;
    if (timed) {
        while (o->prof_ev.size() < o->prof_used + 2) {
            cudaEvent_t e;
            CU(cudaEventCreate(&e));
            o->prof_ev.push_back(e);
        }
        e0 = o->prof_ev[o->prof_used];
        e1 = o->prof_ev[o->prof_used + 1];
        o->prof_used += 2;
        CU(cudaEventRecord(e0, o->stream));
    }
    if (coop)
        CU(cudaLaunchCooperativeKernel(fn, dim3((unsigned)blocks), dim3(kBlock), args, smem, o->stream));
    else
        CU(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(kBlock), args, smem, o->stream));
    if (timed) CU(cudaEventRecord(e1, o->stream));
    ++o->launches;
    ++o->path_launches;
    return BAP_OK;
}

// Sum of the recorded path-kernel event pairs (call after the stream is synchronized).
double prof_collect(bap_option* o) {
    double tot = 0;
    for (size_t i = 0; i + 1 < o->prof_used; i += 2) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, o->prof_ev[i], o->prof_ev[i + 1]) == cudaSuccess) tot += ms;
    }
    o->prof_used = 0;
    return tot;
}

// Phases of a fit, named as in the paper's time distributions: [glp] lattice and point set-up,
// [calc] continuation values (Newton passes, CMC labels), [reg] / [class] the boundary fit or
// the boosting.  Each phase is an NVTX range on the enqueuing host thread and, with profiling
// on (and not inside a graph capture), a pair of CUDA events on the option's stream.
enum Phase : int { PH_GLP = 0, PH_CALC = 1, PH_FIT = 2 };
const char* const kPhaseName[3] = {"[glp]", "[calc]", "[reg/class]"};

int phase_begin(bap_option* o, int phase) {
    nvtxRangePushA(kPhaseName[phase]);
    if (!o->profiling || o->capturing) return -1;
    if (o->phase_ev.size() <= o->phase_used) {
        bap_option::PhaseMark pm{phase, nullptr, nullptr};
        if (cudaEventCreate(&pm.a) != cudaSuccess || cudaEventCreate(&pm.b) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        o->phase_ev.push_back(pm);
    }
    const int i = (int)o->phase_used++;
    o->phase_ev[i].phase = phase;
    cudaEventRecord(o->phase_ev[i].a, o->stream);
    return i;
}

void phase_end(bap_option* o, int i) {
    nvtxRangePop();
    if (i >= 0) cudaEventRecord(o->phase_ev[i].b, o->stream);
}

// Sums the recorded phases of the last fit (after the stream reached them).
void phase_collect(bap_option* o) {
    for (double& v : o->fit_phase_ms) v = 0.0;
    for (size_t i = 0; i < o->phase_used; ++i) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, o->phase_ev[i].a, o->phase_ev[i].b) == cudaSuccess)
            o->fit_phase_ms[o->phase_ev[i].phase] += ms;
    }
    o->phase_used = 0;
}

void base_args(bap_option* o, PathArgs& a, int m, int mode, bool fp64) {
    memset(&a, 0, sizeof a);
    a.model = o->dmodel.as<DevModel>();
    a.n_items = o->n_items;
    a.checks = o->check_buf.as<unsigned long long>();
    a.m = m;
    a.mode = mode;
    a.n_dates = o->n_dates;
    a.payoff = o->payoff;
    a.uniform = o->hm.uniform_dates;
    a.r = o->r;
    a.K = o->K;
    const int d = o->d;
    for (int q = 0; q < d; ++q) {
        for (int j = 0; j <= q; ++j) {
            const double l = o->hm.L[q * MAXD + j];
            a.Lf[q * (q + 1) / 2 + j] = (float)(a.uniform ? o->hm.vol2[1][q] * l : l);
        }
        a.driftf[q] = (float)o->hm.drift2[1][q];
        a.wf[q] = (float)o->hm.w[q];
    }
    a.total_steps = o->total_steps.as<unsigned long long>();
    a.rule_kind = o->rule_kind;
    a.fitted = o->fitted.as<int>();
    if (o->rule_kind == R_IZ) {
        a.rule_src = fp64 ? (const void*)o->coef_d.p : (const void*)o->coef_f.p;
        a.rule_stride = o->n_bnd * iz_stride(o->d, o->degree);
        a.n_bnd = o->n_bnd;
        a.n_coef = iz_stride(o->d, o->degree);
    } else if (o->rule_kind == R_CMC) {
        a.rule_src = fp64 ? (const void*)o->rec_d.p : (const void*)o->rec_f.p;
        a.rule_stride = o->rec_len;
    }
}

bap_status set_rule_iz(bap_option* o, int degree) {
    const int s = o->d - 1;
    if (s == 0) degree = 0;
    o->rule_kind = R_IZ;
    o->n_bnd = (o->payoff == BAP_MAX_CALL && o->d > 1) ? o->d : 1;
    o->degree = degree;
    o->n_coef = n_basis(s, degree);
    const size_t nc = (size_t)(o->n_dates + 1) * o->n_bnd * o->n_coef;
    const size_t ns = (size_t)(o->n_dates + 1) * o->n_bnd * iz_stride(o->d, degree);
    TRY(o->coef64.reserve(nc * 8));
    TRY(o->coef_f.reserve(ns * 4));
    TRY(o->coef_d.reserve(ns * 8));
    CU(cudaMemsetAsync(o->coef64.p, 0, nc * 8, o->stream));
    CU(cudaMemsetAsync(o->coef_f.p, 0, ns * 4, o->stream));
    CU(cudaMemsetAsync(o->coef_d.p, 0, ns * 8, o->stream));
    CU(cudaMemsetAsync(o->fitted.p, 0, (o->n_dates + 1) * sizeof(int), o->stream));
    return BAP_OK;
}

bap_status set_rule_cmc(bap_option* o, int max_stumps) {
    o->rule_kind = R_CMC;
    o->max_stumps = max_stumps;
    o->rec_len = cmc_record_len(o->d + 1, max_stumps);
    const size_t nd = o->n_dates + 1;
    TRY(o->n_stumps.reserve(nd * 4));
    TRY(o->feat.reserve(nd * max_stumps * 4));
    TRY(o->thr.reserve(nd * max_stumps * 8));
    TRY(o->pol.reserve(nd * max_stumps * 4));
    TRY(o->alpha.reserve(nd * max_stumps * 8));
    TRY(o->rec_f.reserve(nd * o->rec_len * 4));
    TRY(o->rec_d.reserve(nd * o->rec_len * 8));
    CU(cudaMemsetAsync(o->n_stumps.p, 0, nd * 4, o->stream));
    CU(cudaMemsetAsync(o->feat.p, 0, nd * max_stumps * 4, o->stream));
    CU(cudaMemsetAsync(o->thr.p, 0, nd * max_stumps * 8, o->stream));
    CU(cudaMemsetAsync(o->pol.p, 0, nd * max_stumps * 4, o->stream));
    CU(cudaMemsetAsync(o->alpha.p, 0, nd * max_stumps * 8, o->stream));
    CU(cudaMemsetAsync(o->rec_f.p, 0, nd * o->rec_len * 4, o->stream));
    CU(cudaMemsetAsync(o->rec_d.p, 0, nd * o->rec_len * 8, o->stream));
    CU(cudaMemsetAsync(o->fitted.p, 0, nd * sizeof(int), o->stream));
    return BAP_OK;
}

// Scratch for n items of N paths each.
// Scratch for n items and `slots` unit partials.
bap_status reserve_items(bap_option* o, int n, long long slots, int max_iter) {
    // the path kernel numbers unit slots in 32 bits
    if (slots >= (1LL << 32)) return fail(BAP_EINVAL, "too many path units (%lld)", slots);
    const int d = o->d;
    TRY(o->start.reserve((size_t)n * d * 8));
    TRY(o->l0f.reserve((size_t)n * d * 4));
    TRY(o->state.reserve((size_t)n * sizeof(ItemState)));
    TRY(o->pivot.reserve((size_t)n * 4));
    TRY(o->ctr_item.reserve((size_t)n * 4));
    TRY(o->active0.reserve((size_t)n * 4));
    TRY(o->active1.reserve((size_t)n * 4));
    TRY(o->counts.reserve((size_t)(max_iter + 2) * 4));
    TRY(o->work.reserve((size_t)(max_iter + 2) * 8));
    TRY(o->partial.reserve((size_t)slots * 3 * 8));
    TRY(o->partial_steps.reserve((size_t)slots * 8));
    TRY(o->done.reserve((size_t)n * 4));
    TRY(o->out_sums.reserve((size_t)n * 3 * 8));
    TRY(o->out_steps.reserve((size_t)n * 8));
    TRY(o->label_y.reserve((size_t)n * 8));
    TRY(o->label.reserve((size_t)n * 4));
    TRY(o->iterstate.reserve(sizeof(IterState)));
    return BAP_OK;
}

__global__ void iota_kernel(int* p, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

bap_status record_diag(bap_option* o, int m, bool iz) {
    const int n = o->n_items;
    const int g = (n + 255) / 256;
    if (iz) {
        collect_points_kernel<<<g, 256, 0, o->stream>>>(
            o->state.as<ItemState>(), n, o->diag_x.as<double>() + (size_t)m * n,
            o->diag_it.as<int>() + (size_t)m * n, o->diag_st.as<int>() + (size_t)m * n,
            o->stat_counts.as<int>());
    } else {
        collect_labels_kernel<<<g, 256, 0, o->stream>>>(
            o->label_y.as<double>(), n, o->diag_x.as<double>() + (size_t)m * n,
            o->diag_it.as<int>() + (size_t)m * n, o->diag_st.as<int>() + (size_t)m * n);
    }
    ++o->launches;
    CU(cudaGetLastError());
    return BAP_OK;
}

// One Newton pass of date m: pass `it` (plain form), or the pass that the iteration state names
// (it < 0: graph form, advanced by newton_decide_kernel).
bap_status enqueue_newton_pass(bap_option* o, const bap_iz_params* p, int m, int it, int chunk,
                               int C) {
    PathArgs a;
    base_args(o, a, m, MODE_NEWTON, false);
    a.rk = make_round_keys(p->seed, P_IZ, (uint32_t)m);
    a.N = p->N1;
    a.chunk = chunk;
    a.C = C;
    a.list[0] = o->active0.as<int>();
    a.list[1] = o->active1.as<int>();
    a.count = o->counts.as<int>();
    a.work = o->work.as<unsigned long long>();
    if (it >= 0) a.pass_it = it;
    else a.iter_ptr = &o->iterstate.as<IterState>()->iter;
    a.start = o->start.as<double>();
    a.l0f = o->l0f.as<float>();
    a.ctr_item = o->ctr_item.as<int>();
    a.pivot = o->pivot.as<int>();
    a.partial = o->partial.as<double>();
    a.partial_steps = o->partial_steps.as<long long>();
    a.done = o->done.as<int>();
    a.state = o->state.as<ItemState>();
    a.f_tol = p->f_tol;
    a.x_tol = p->x_tol;
    a.fp_eps = p->fp_eps;
    a.max_iter = p->max_iter;
    a.fixed_point = p->fixed_point;
    set_tail_split(o, a);
    return launch_path(o, a, R_IZ, false, (long long)o->n_items * std::max(C, a.C_tail));
}

// All Newton passes of date m in one cooperative launch (newton_coop_kernel), on the per-pass
// lists, counts and unit counters of the plain form; the grid barrier's counter is the last
// count slot (index max_iter + 1, which no pass writes) and its failure flag stat_counts[3].
bap_status enqueue_newton_coop(bap_option* o, const bap_iz_params* p, int m, int chunk, int C) {
    PathArgs a;
    base_args(o, a, m, MODE_NEWTON, false);
    a.rk = make_round_keys(p->seed, P_IZ, (uint32_t)m);
    a.N = p->N1;
    a.chunk = chunk;
    a.C = C;
    a.list[0] = o->active0.as<int>();
    a.list[1] = o->active1.as<int>();
    a.count = o->counts.as<int>();
    a.work = o->work.as<unsigned long long>();
    a.passes = o->stat_counts.as<int>() + 2;
    a.coop_bar = reinterpret_cast<unsigned*>(o->counts.as<int>() + p->max_iter + 1);
    a.coop_err = o->stat_counts.as<int>() + 3;
    // a wait at the barrier never lasts longer than a pass: allow 5 s plus 1 ns per path step
    a.coop_limit_ns = o->wait_limit_ns != 0
                          ? o->wait_limit_ns
                          : 5000000000ULL + (unsigned long long)o->n_items *
                                                (unsigned long long)p->N1 * (unsigned long long)(o->n_dates - m);
    a.start = o->start.as<double>();
    a.l0f = o->l0f.as<float>();
    a.ctr_item = o->ctr_item.as<int>();
    a.pivot = o->pivot.as<int>();
    a.partial = o->partial.as<double>();
    a.partial_steps = o->partial_steps.as<long long>();
    a.done = o->done.as<int>();
    a.state = o->state.as<ItemState>();
    a.f_tol = p->f_tol;
    a.x_tol = p->x_tol;
    a.fp_eps = p->fp_eps;
    a.max_iter = p->max_iter;
    a.fixed_point = p->fixed_point;
    set_tail_split(o, a);
    return launch_path(o, a, R_NEWTON_COOP, false, (long long)o->n_items * std::max(C, a.C_tail));
}

bap_status enqueue_iz_prologue(bap_option* o, const bap_iz_params* p) {
    const int n = o->n_items, J = p->J, s = o->d - 1;
    cudaStream_t st = o->stream;
    CU(cudaMemsetAsync(o->diag_x.p, 0, (size_t)(o->n_dates + 1) * n * 8, st));
    CU(cudaMemsetAsync(o->diag_it.p, 0, (size_t)(o->n_dates + 1) * n * 4, st));
    CU(cudaMemsetAsync(o->diag_st.p, 0, (size_t)(o->n_dates + 1) * n * 4, st));
    CU(cudaMemsetAsync(o->done.p, 0, (size_t)n * 4, st));
    CU(cudaMemsetAsync(o->total_steps.p, 0, 8, st));
    CU(cudaMemsetAsync(o->stat_counts.p, 0, 16, st));
    iota_kernel<<<(n + 255) / 256, 256, 0, st>>>(o->ctr_item.as<int>(), n);
    ++o->launches;
    if (s >= 2 && J > 2) {
        const int warps = J - 1;
        korobov_merit_kernel<<<(warps * 32 + 255) / 256, 256, 0, st>>>(J, s, o->merit.as<double>());
        ++o->launches;
    }
    korobov_pick_kernel<<<1, 256, 0, st>>>(J, s, o->merit.as<double>(), o->korobov_a.as<int>());
    ++o->launches;
    CU(cudaGetLastError());
    return BAP_OK;
}

bap_status enqueue_iz_setup(bap_option* o, const bap_iz_params* p, int m, bool device_loop) {
    cudaStream_t st = o->stream;
    if (device_loop) CU(cudaMemsetAsync(o->iterstate.p, 0, sizeof(IterState), st));
    CU(cudaMemsetAsync(o->counts.p, 0, (size_t)(p->max_iter + 2) * 4, st));
    CU(cudaMemsetAsync(o->work.p, 0, (size_t)(p->max_iter + 2) * 8, st));
    int* count0 = o->counts.as<int>();
    iz_setup_kernel<<<(o->n_items + 127) / 128, 128, 0, st>>>(
        o->dmodel.as<DevModel>(), m, p->J, o->n_bnd, o->korobov_a.as<int>(), o->start.as<double>(),
        o->state.as<ItemState>(), o->pivot.as<int>(), o->active0.as<int>(), count0,
        o->coef64.as<double>(), o->n_coef, o->degree, o->fitted.as<int>(), p->warm_start,
        o->l0f.as<float>());
    ++o->launches;
    CU(cudaGetLastError());
    return BAP_OK;
}

bap_status enqueue_iz_fit_date_end(bap_option* o, const bap_iz_params* p, int m) {
    ls_fit_kernel<<<o->n_bnd, kLsThreads, 0, o->stream>>>(
        o->dmodel.as<DevModel>(), m, p->J, o->n_bnd, o->degree, o->n_coef, o->start.as<double>(),
        o->state.as<ItemState>(), o->coef64.as<double>(), o->coef_f.as<float>(),
        o->coef_d.as<double>(), o->fitted.as<int>());
    ++o->launches;
    CU(cudaGetLastError());
    return record_diag(o, m, true);
}

// The whole I&Z fit as one graph: per date the item set-up, a conditional while node whose body
// is one Newton pass followed by newton_decide_kernel, then the regression and diagnostics.
bap_status build_iz_graph(bap_option* o, const bap_iz_params* p, int chunk, int C) {
    cudaGraph_t g = nullptr;
    CU(cudaGraphCreate(&g, 0));
    cudaStream_t st = o->stream;
    o->capturing = 1;
    bap_status status = BAP_OK;
    auto abort_capture = [&]() {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(st, &junk);
        if (junk && junk != g) cudaGraphDestroy(junk);
    };
    cudaError_t e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        o->capturing = 0;
        cudaGraphDestroy(g);
        return fail(BAP_ECUDA, "capture: %s", cudaGetErrorString(e));
    }
    status = enqueue_iz_prologue(o, p);
    for (int m = o->n_dates - 1; m >= 1 && status == BAP_OK; --m) {
        status = enqueue_iz_setup(o, p, m, true);
        if (status != BAP_OK) break;
        // frontier of the capture so far
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
        std::vector<cudaGraphNode_t> frontier(deps, deps + ndeps);
        cudaGraph_t gg = nullptr;
        if (e == cudaSuccess) e = cudaStreamEndCapture(st, &gg);
        if (e != cudaSuccess) { status = fail(BAP_ECUDA, "capture: %s", cudaGetErrorString(e)); break; }
        cudaGraphConditionalHandle h;
        e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t wnode = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, g, frontier.data(), nullptr, frontier.size(), &np);
        if (e != cudaSuccess) { status = fail(BAP_ECUDA, "conditional node: %s", cudaGetErrorString(e)); break; }
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { status = fail(BAP_ECUDA, "capture: %s", cudaGetErrorString(e)); break; }
        status = enqueue_newton_pass(o, p, m, -1, chunk, C);
        if (status == BAP_OK) {
            newton_decide_kernel<<<1, 32, 0, st>>>(o->iterstate.as<IterState>(), o->counts.as<int>(),
                                                   p->max_iter, h, o->stat_counts.as<int>() + 2);
            ++o->launches;
            if (cudaGetLastError() != cudaSuccess) status = fail(BAP_ECUDA, "decide kernel");
        }
        cudaGraph_t bb = nullptr;
        e = cudaStreamEndCapture(st, &bb);
        if (status != BAP_OK) break;
        if (e != cudaSuccess) { status = fail(BAP_ECUDA, "capture: %s", cudaGetErrorString(e)); break; }
        e = cudaStreamBeginCaptureToGraph(st, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { status = fail(BAP_ECUDA, "capture: %s", cudaGetErrorString(e)); break; }
        status = enqueue_iz_fit_date_end(o, p, m);
    }
    if (status != BAP_OK) {
        abort_capture();
        o->capturing = 0;
        cudaGraphDestroy(g);
        return status;
    }
    cudaGraph_t gend = nullptr;
    e = cudaStreamEndCapture(st, &gend);
    o->capturing = 0;
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(BAP_ECUDA, "capture end: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(BAP_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    o->graph_exec = ex;
    o->graph_params = *p;
    o->graph_chunk = chunk;
    return BAP_OK;
}

bool same_iz(const bap_iz_params& a, const bap_iz_params& b) {
    return a.J == b.J && a.N1 == b.N1 && a.f_tol == b.f_tol && a.x_tol == b.x_tol &&
           a.max_iter == b.max_iter && a.degree == b.degree && a.seed == b.seed &&
           a.fixed_point == b.fixed_point && a.fp_eps == b.fp_eps && a.warm_start == b.warm_start;
}

bap_status run_sums_enqueue(bap_option* o, int m, int mode, bool fp64, const RoundKeys& rk,
                            int n_items, long long N, const int* d_item_ids, const int* d_pivots,
                            double* d_start, double* d_out_sums, long long* d_out_steps) {
    const int chunk = choose_chunk(n_items, N);
    const int C = (int)((N + chunk - 1) / chunk);
    TRY(o->partial.reserve((size_t)n_items * C * 3 * 8));
    TRY(o->partial_steps.reserve((size_t)n_items * C * 8));
    TRY(o->done.reserve((size_t)n_items * 4));
    TRY(o->work.reserve(16));
    TRY(o->counts.reserve(16));
    cudaStream_t st = o->stream;
    CU(cudaMemsetAsync(o->done.p, 0, (size_t)n_items * 4, st));
    CU(cudaMemsetAsync(o->work.p, 0, 8, st));
    CU(cudaMemsetAsync(o->total_steps.p, 0, 8, st));
    set_int_kernel<<<1, 32, 0, st>>>(o->counts.as<int>(), n_items);
    ++o->launches;
    PathArgs a;
    base_args(o, a, m, mode, fp64);
    a.n_items = n_items;
    a.rk = rk;
    a.N = N;
    a.chunk = chunk;
    a.C = C;
    a.count = o->counts.as<int>();
    a.work = o->work.as<unsigned long long>();
    a.start = d_start;
    a.ctr_item = d_item_ids;
    a.pivot = d_pivots;
    a.partial = o->partial.as<double>();
    a.partial_steps = o->partial_steps.as<long long>();
    a.done = o->done.as<int>();
    a.out_sums = d_out_sums;
    a.out_steps = d_out_steps;
    a.trace_tau = o->trace_tau.as<int>();
    a.trace_phi = o->trace_phi.as<double>();
    return launch_path(o, a, o->rule_kind, fp64, (long long)n_items * C);
}

bap_status run_sums(bap_option* o, int m, int mode, bool fp64, const RoundKeys& rk, int n_items,
                    long long N, const int* d_item_ids, const int* d_pivots, double* d_start,
                    double* h_sums, long long* h_steps) {
    TRY(o->out_sums.reserve((size_t)n_items * 3 * 8));
    TRY(o->out_steps.reserve((size_t)n_items * 8));
    TRY(run_sums_enqueue(o, m, mode, fp64, rk, n_items, N, d_item_ids, d_pivots, d_start,
                         o->out_sums.as<double>(), o->out_steps.as<long long>()));
    cudaStream_t st = o->stream;
    CU(cudaMemcpyAsync(h_sums, o->out_sums.p, (size_t)n_items * 3 * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(h_steps, o->out_steps.p, (size_t)n_items * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return BAP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Building blocks shared with the serving loop.

namespace bap {

// Validated model and its FP64 set-up: the lower Cholesky factor of rho (the positive
// definiteness check) and the per-date stepping constants in log2 units.  A few hundred flops
// per option, done once on the host so that creating an option never waits for the device.
bap_status model_prepare(const bap_model* md, DevModel* out) {
    if (!md || !out) return fail(BAP_EINVAL, "null argument");
    const int d = md->d;
    if (d < 1 || d > BAP_MAX_D) return fail(BAP_EINVAL, "d=%d outside 1..%d", d, BAP_MAX_D);
    if (!md->S0 || !md->sigma || !md->delta || !md->rho) return fail(BAP_EINVAL, "null model array");
    if (!(md->K > 0) || !(md->T > 0)) return fail(BAP_EINVAL, "K and T must be positive");
    if (md->n_dates < 1 || md->n_dates > BAP_MAX_DATES)
        return fail(BAP_EINVAL, "n_dates=%d outside 1..%d", md->n_dates, BAP_MAX_DATES);
    if (md->payoff < BAP_MAX_CALL || md->payoff > BAP_GEO_CALL) return fail(BAP_EINVAL, "bad payoff");
    if (!std::isfinite(md->r)) return fail(BAP_EINVAL, "bad rate");
    for (int q = 0; q < d; ++q) {
        if (!(md->S0[q] > 0) || !std::isfinite(md->S0[q])) return fail(BAP_EINVAL, "S0[%d] must be positive", q);
        if (!(md->sigma[q] > 0) || !std::isfinite(md->sigma[q])) return fail(BAP_EINVAL, "sigma[%d] must be positive", q);
        if (!std::isfinite(md->delta[q])) return fail(BAP_EINVAL, "bad delta[%d]", q);
        if (md->weights && !(md->weights[q] > 0)) return fail(BAP_EINVAL, "weights must be positive");
        for (int j = 0; j < d; ++j) {
            const double v = md->rho[q * d + j];
            if (!std::isfinite(v) || std::fabs(v - md->rho[j * d + q]) > 1e-12 || std::fabs(v) > 1.0 + 1e-12)
                return fail(BAP_EINVAL, "rho must be a symmetric correlation matrix");
        }
        if (std::fabs(md->rho[q * d + q] - 1.0) > 1e-12) return fail(BAP_EINVAL, "rho must have a unit diagonal");
    }
    DevModel hm{};
    hm.d = d;
    hm.n_dates = md->n_dates;
    hm.payoff = md->payoff;
    hm.r = md->r;
    hm.K = md->K;
    for (int q = 0; q < d; ++q) {
        hm.S0[q] = md->S0[q];
        hm.sigma[q] = md->sigma[q];
        hm.delta[q] = md->delta[q];
        hm.w[q] = md->weights ? md->weights[q] : 1.0 / d;
    }
    hm.t[0] = 0.0;
    for (int k = 1; k <= md->n_dates; ++k) {
        hm.t[k] = md->dates ? md->dates[k - 1] : md->T * k / md->n_dates;
        if (!(hm.t[k] > hm.t[k - 1])) return fail(BAP_EINVAL, "dates must increase from 0");
    }
    if (std::fabs(hm.t[md->n_dates] - md->T) > 1e-12 * md->T) return fail(BAP_EINVAL, "last date must equal T");
    hm.t[md->n_dates] = md->T;
    // Cholesky rho = L L^T (lower, FP64)
    for (int j = 0; j < d; ++j) {
        double sjj = md->rho[j * d + j];
        for (int k = 0; k < j; ++k) sjj -= hm.L[j * MAXD + k] * hm.L[j * MAXD + k];
        if (!(sjj > 1e-14)) return fail(BAP_EINVAL, "rho is not positive definite");
        const double ljj = std::sqrt(sjj);
        hm.L[j * MAXD + j] = ljj;
        for (int i = j + 1; i < d; ++i) {
            double v = md->rho[i * d + j];
            for (int k = 0; k < j; ++k) v -= hm.L[i * MAXD + k] * hm.L[j * MAXD + k];
            hm.L[i * MAXD + j] = v / ljj;
        }
    }
    const double inv_ln2 = 1.4426950408889634;
    int uniform = 1;
    const double dt1 = hm.t[1] - hm.t[0];
    for (int k = 1; k <= hm.n_dates; ++k) {
        const double dt = hm.t[k] - hm.t[k - 1];
        if (std::fabs(dt - dt1) > 1e-12 * hm.t[hm.n_dates]) uniform = 0;
        for (int q = 0; q < d; ++q) {
            hm.drift2[k][q] = (hm.r - hm.delta[q] - 0.5 * hm.sigma[q] * hm.sigma[q]) * dt * inv_ln2;
            hm.vol2[k][q] = hm.sigma[q] * std::sqrt(dt) * inv_ln2;
        }
    }
    hm.uniform_dates = uniform;
    *out = hm;
    return BAP_OK;
}

// CUDA loads a kernel on its first use, and that load waits for the work already running on
// the device: under concurrent requests a first use stalled the calling thread for up to a
// second.  So all kernels of the library are loaded (and the shared-memory limits of those that
// need more than the default raised) once per device, when the first option or server is made.
bap_status preload_kernels(int device) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), device) != done.end()) return BAP_OK;
    {
        std::lock_guard<std::mutex> lk2(g_fn_mu);
        for (int D = 1; D <= MAXD; ++D) {
            for (int rule : {(int)R_NONE, (int)R_IZ, (int)R_CMC, R_NEWTON_COOP, R_IZ3, R_NEWTON_COOP3}) {
                const bool coop = rule == R_NEWTON_COOP || rule == R_NEWTON_COOP3;
                for (int fp64 = 0; fp64 < (coop ? 1 : 2); ++fp64) {
                    for (int ppl = 1; ppl <= 2; ++ppl) {
                        for (int pay = -1; pay <= 2; ++pay) {
                            const void* fn = path_fn(D, rule, fp64 != 0, ppl, pay);
                            if (!fn) continue;    // no cubic kernels above MAXD_CUBIC
                            TRY(raise_smem_limit(fn, device, g_fn[{fn, device}]));
                        }
                    }
                }
            }
        }
        for (const void* ab : {(const void*)adaboost_kernel, (const void*)adaboost_warp_kernel})
            TRY(raise_smem_limit(ab, device, g_fn[{ab, device}]));
        // the cluster boosting kernels: d + 1 features up to 11 blocks per cluster, above the
        // portable 8
        for (const void* fn : {(const void*)adaboost_cluster_kernel, (const void*)logitboost_cluster_kernel}) {
            TRY(raise_smem_limit(fn, device, g_fn[{fn, device}]));
            CU(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        }
    }
    const void* others[] = {
        (const void*)iota_kernel,          (const void*)korobov_merit_kernel,
        (const void*)korobov_pick_kernel,  (const void*)iz_setup_kernel,
        (const void*)stage_iz_kernel,      (const void*)ls_fit_kernel,
        (const void*)train_points_kernel,  (const void*)stage_cmc_kernel,
        (const void*)newton_decide_kernel, (const void*)set_int_kernel,
        (const void*)rng_debug_kernel,     (const void*)collect_points_kernel,
        (const void*)collect_labels_kernel};
    for (const void* fn : others) {
        cudaFuncAttributes fa;
        CU(cudaFuncGetAttributes(&fa, fn));
    }
    done.push_back(device);
    return BAP_OK;
}

// Stream, events and page-locked results of an option, without a model yet.
bap_status option_alloc(bap_option** out) {
    *out = nullptr;
    int dev;
    if (!has_device(&dev)) return fail(BAP_ECUDA, "no CUDA device");
    TRY(preload_kernels(dev));
    bap_option* o = new (std::nothrow) bap_option();
    if (!o) return fail(BAP_ENOMEM, "host allocation");
    o->device = dev;
    keep_pool_cached(dev);
    cudaError_t e = cudaDeviceGetAttribute(&o->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&o->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        option_destroy(o);
        return fail(BAP_ECUDA, "%s", cudaGetErrorString(e));
    }
    o->stream = o->own_stream;
    if (cudaEventCreate(&o->ev0) != cudaSuccess || cudaEventCreate(&o->ev1) != cudaSuccess ||
        cudaEventCreate(&o->ev2) != cudaSuccess || cudaEventCreate(&o->ev3) != cudaSuccess) {
        option_destroy(o);
        return fail(BAP_ECUDA, "event create");
    }
    o->pin = pinned_get();
    if (!o->pin) {
        option_destroy(o);
        return fail(BAP_ENOMEM, "page-locked host allocation");
    }
    memset(o->pin, 0, sizeof(PinnedOut));
    *out = o;
    return BAP_OK;
}

// Gives an idle option a (prepared) model: uploads it and clears the fitted rule.
bap_status option_load(bap_option* o, const DevModel& hm) {
    AllocScope scope(o->stream);
    o->d = hm.d;
    o->n_dates = hm.n_dates;
    o->payoff = hm.payoff;
    o->r = hm.r;
    o->K = hm.K;
    o->T = hm.t[hm.n_dates];
    o->hm = hm;
    o->rule_kind = R_NONE;
    o->method = -1;
    o->n_items = 0;
    o->last_noconv = o->last_noroot = 0;
    o->last_fit_steps = 0;
    o->last_fit_ms = 0;
    o->fit_launches = o->fit_path_launches = 0;
    o->fit_path_ms = 0;
    if (o->graph_exec) {
        cudaGraphExecDestroy(o->graph_exec);
        o->graph_exec = nullptr;
    }
    TRY(o->dmodel.reserve(sizeof(DevModel)));
    TRY(o->s0buf.reserve((size_t)MAXD * 8));
    TRY(o->fitted.reserve((MAXDATES + 1) * sizeof(int)));
    TRY(o->total_steps.reserve(8));
    TRY(o->stat_counts.reserve(16));
    TRY(o->one.reserve(8));
    TRY(o->check_buf.reserve(16));
    CU(cudaMemsetAsync(o->check_buf.p, 0, 16, o->stream));
    CU(cudaMemcpyAsync(o->dmodel.p, &o->hm, sizeof(DevModel), cudaMemcpyHostToDevice, o->stream));
    CU(cudaMemcpyAsync(o->s0buf.p, o->hm.S0, (size_t)hm.d * 8, cudaMemcpyHostToDevice, o->stream));
    CU(cudaMemsetAsync(o->fitted.p, 0, (hm.n_dates + 1) * sizeof(int), o->stream));
    return BAP_OK;
}

bap_status option_create(const bap_model* md, bap_option** out) {
    if (!out) return fail(BAP_EINVAL, "null argument");
    *out = nullptr;
    DevModel hm;
    TRY(model_prepare(md, &hm));
    bap_option* o;
    TRY(option_alloc(&o));
    const bap_status st = option_load(o, hm);
    if (st != BAP_OK) {
        option_destroy(o);
        return st;
    }
    *out = o;
    return BAP_OK;
}

void option_destroy(bap_option* o) {
    if (!o) return;
    if (o->stream) cudaStreamSynchronize(o->stream);
    // the option is idle: return its memory to the pool in the order of its own stream
    cudaStream_t own = o->own_stream;
    o->for_each_buf([&](DevBuf& b) { b.release(own); });
    for (cudaEvent_t e : o->prof_ev) cudaEventDestroy(e);
    if (o->graph_exec) cudaGraphExecDestroy(o->graph_exec);
    if (o->ev0) cudaEventDestroy(o->ev0);
    if (o->ev1) cudaEventDestroy(o->ev1);
    if (o->ev2) cudaEventDestroy(o->ev2);
    if (o->ev3) cudaEventDestroy(o->ev3);
    pinned_put(o->pin);
    delete o;
    if (own) cudaStreamDestroy(own);
}

bap_status validate_iz(int d, const bap_iz_params* p) {
    if (!p) return fail(BAP_EINVAL, "null argument");
    if (p->J < 1 || p->J > 8192) return fail(BAP_EINVAL, "J=%d outside 1..8192", p->J);
    if (p->N1 < 1 || p->N1 > (1LL << 31)) return fail(BAP_EINVAL, "N1 outside 1..2^31");
    if (p->max_iter < 1 || p->max_iter > 200) return fail(BAP_EINVAL, "max_iter outside 1..200");
    if (p->degree < 0 || p->degree > 3) return fail(BAP_EINVAL, "degree outside 0..3");
    if (p->degree == 3 && d > MAXD_CUBIC)
        return fail(BAP_EINVAL, "cubic boundaries need d <= %d", MAXD_CUBIC);
    if (!(p->f_tol >= 0) || !(p->x_tol >= 0)) return fail(BAP_EINVAL, "negative tolerance");
    if (p->fixed_point && !(p->fp_eps > 0)) return fail(BAP_EINVAL, "fp_eps must be positive");
    if (p->warm_start != 0 && p->warm_start != 1) return fail(BAP_EINVAL, "warm_start outside 0..1");
    return BAP_OK;
}

bap_status validate_cmc(const bap_option* o, const bap_cmc_params* p) {
    (void)o;
    if (!p) return fail(BAP_EINVAL, "null argument");
    if (p->J < 2 || p->J > 8192) return fail(BAP_EINVAL, "J=%d outside 2..8192", p->J);
    if (p->N2 < 1 || p->N2 > (1LL << 31)) return fail(BAP_EINVAL, "N2 outside 1..2^31");
    if (p->n_stumps < 1 || p->n_stumps > BAP_MAX_STUMPS) return fail(BAP_EINVAL, "n_stumps outside 1..%d", BAP_MAX_STUMPS);
    if (p->sampler != 0 && p->sampler != 1) return fail(BAP_EINVAL, "sampler outside 0..1");
    if (p->boost != 0 && p->boost != 1) return fail(BAP_EINVAL, "boost outside 0..1");
    if (p->boost == 1 && (p->n_stumps > BAP_MAX_STUMPS / 2 || p->J > 4096))
        return fail(BAP_EINVAL, "LogitBoost: rounds 1..%d and J <= 4096", BAP_MAX_STUMPS / 2);
    return BAP_OK;
}

bap_status validate_price(const bap_option* o, int64_t n_paths) {
    if (!o) return fail(BAP_EINVAL, "null argument");
    if (n_paths < 2 || n_paths > (1LL << 40)) return fail(BAP_EINVAL, "n_paths outside 2..2^40");
    return BAP_OK;
}

bap_status enqueue_fit_iz(bap_option* o, const bap_iz_params* p) {
    AllocScope scope(o->stream);
    o->launches = o->path_launches = 0;
    o->prof_used = 0;
    o->phase_used = 0;
    TRY(set_rule_iz(o, p->degree));
    o->method = 0;
    if (o->n_dates < 2) {
        o->n_items = 0;
        memset(o->pin, 0, sizeof(PinnedOut));
        CU(cudaEventRecord(o->ev0, o->stream));
        CU(cudaEventRecord(o->ev1, o->stream));
        return BAP_OK;
    }
    const int J = p->J;
    const int n = o->n_bnd * J;
    o->n_items = n;
    const LaunchChoice lc = tuned_launch(o->d, tune_kind(BAP_METHOD_IZ, p->degree), n, p->N1);
    const int chunk = choose_chunk(n, p->N1, o->unit_paths ? o->unit_paths : lc.unit);
    const int C = (int)((p->N1 + chunk - 1) / chunk);
    o->ppl_fit = lc.ppl;
    o->last_unit = chunk;
    TRY(reserve_items(o, n, newton_unit_slots(n, p->N1, chunk, o->sm_count), p->max_iter));
    TRY(o->korobov_a.reserve(8));
    TRY(o->merit.reserve((size_t)(J + 1) * 8));
    TRY(o->diag_x.reserve((size_t)(o->n_dates + 1) * n * 8));
    TRY(o->diag_it.reserve((size_t)(o->n_dates + 1) * n * 4));
    TRY(o->diag_st.reserve((size_t)(o->n_dates + 1) * n * 4));
    cudaStream_t st = o->stream;
    bool use_graph = o->launch_mode == LAUNCH_GRAPH && !o->graph_failed && !o->profiling;
    if (use_graph && (!o->graph_exec || !same_iz(o->graph_params, *p) || o->graph_chunk != chunk)) {
        if (o->graph_exec) {
            cudaGraphExecDestroy(o->graph_exec);
            o->graph_exec = nullptr;
        }
        const long long saved = o->launches, saved_p = o->path_launches;
        if (build_iz_graph(o, p, chunk, C) != BAP_OK) {
            o->graph_failed = 1;     // this device or driver cannot run it: use the plain form
            use_graph = false;
            cudaGetLastError();
        }
        o->launches = saved;
        o->path_launches = saved_p;
    }
    CU(cudaEventRecord(o->ev0, st));
    o->last_graph = use_graph ? 1 : 0;
    if (use_graph) {
        CU(cudaGraphLaunch(o->graph_exec, st));
        // kernels in the graph: prologue (iota, lattice) + per date (set-up, LS, diagnostics);
        // the Newton passes actually run (a path kernel and a decide kernel each) are counted on
        // the device and added by finish_fit_iz
        o->launches += 2 + (p->J > 2 && o->d >= 3) + 3LL * (o->n_dates - 1);
    } else {
        int ph = phase_begin(o, PH_GLP);
        bap_status st = enqueue_iz_prologue(o, p);
        phase_end(o, ph);
        TRY(st);
        for (int m = o->n_dates - 1; m >= 1; --m) {
            ph = phase_begin(o, PH_GLP);
            st = enqueue_iz_setup(o, p, m, false);
            phase_end(o, ph);
            TRY(st);
            ph = phase_begin(o, PH_CALC);
            if (o->launch_mode == LAUNCH_COOP) {
                st = enqueue_newton_coop(o, p, m, chunk, C);
            } else {
                for (int it = 0; it < p->max_iter && st == BAP_OK; ++it)
                    st = enqueue_newton_pass(o, p, m, it, chunk, C);
            }
            phase_end(o, ph);
            TRY(st);
            ph = phase_begin(o, PH_FIT);
            st = enqueue_iz_fit_date_end(o, p, m);
            phase_end(o, ph);
            TRY(st);
        }
    }
    CU(cudaEventRecord(o->ev1, st));
    CU(cudaMemcpyAsync(&o->pin->fit_steps, o->total_steps.p, 8, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(o->pin->counts, o->stat_counts.p, 16, cudaMemcpyDeviceToHost, st));
    return BAP_OK;
}

bap_status finish_fit_iz(bap_option* o) {
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, o->ev0, o->ev1));
    o->last_fit_ms = ms;
    o->last_fit_steps = (long long)o->pin->fit_steps;
    o->last_noconv = o->pin->counts[0];
    o->last_noroot = o->pin->counts[1];
    if (o->pin->counts[3] != 0)
        return fail(BAP_ECUDA, "Newton loop: a grid barrier of the cooperative launch timed out");
    if (o->last_graph) {
        o->launches += 2LL * o->pin->counts[2];
        o->path_launches += o->pin->counts[2];
    }
    o->fit_launches = o->launches;
    o->fit_path_launches = o->path_launches;
    o->fit_path_ms = prof_collect(o);
    phase_collect(o);
    return o->last_noconv > 0 ? BAP_ENOCONV : BAP_OK;
}

// Threads per block of the cluster boosting kernels for J points: 1024 above J = 2048 (shorter
// per-thread scans), else 512 (measured faster at J = 1024).  The stumps do not depend on it.
int cluster_boost_threads(int J) { return J > 2048 ? kClusterBoostThreads : kClusterBoostThreads / 2; }

// Launch configuration of the cluster boosting kernels: one cluster of nF blocks.
void boost_cluster_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int nF, size_t smem,
                          cudaStream_t st, int threads) {
    cfg.gridDim = dim3((unsigned)nF);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)nF;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

// Whether a cluster of nF blocks of this boosting kernel fits on the device (cached per kernel,
// device, nF and size).
bap_status boost_cluster_fits(const void* fn, int device, int nF, size_t smem, int threads,
                              cudaStream_t st, bool* ok) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, size_t, int>, bool> known;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(fn, device, nF, smem, threads);
    auto it = known.find(key);
    if (it == known.end()) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        boost_cluster_config(cfg, attr, nF, smem, st, threads);
        int n = 0;
        const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
        if (e != cudaSuccess) cudaGetLastError();
        it = known.emplace(key, e == cudaSuccess && n >= 1).first;
    }
    *ok = it->second;
    return BAP_OK;
}

// How the boosting of a J-point CMC date runs: the kernel form and its shared memory.
struct BoostPlan {
    bool logit = false, warp_form = false, cluster = false;
    int cl_threads = 0;
    size_t ab_smem = 0, abc_smem = 0, abw_smem = 0, lb_smem = 0;
};

bap_status boost_plan(bap_option* o, const bap_cmc_params* p, BoostPlan* bp) {
    const int J = p->J, nF = o->d + 1;
    cudaStream_t st = o->stream;
    BoostPlan& b = *bp;
    b.logit = p->boost == 1;
    int P2 = 1;
    while (P2 < J) P2 <<= 1;
    b.ab_smem = (size_t)J * 8 + std::max((size_t)P2 * 12, (size_t)J * 8) + (size_t)J + 16;
    // the cluster form (one block per feature) when asked for and the device can place it
    b.abc_smem = (size_t)J * 10 + std::max((size_t)P2 * 12, (size_t)J * 16) + 4 +
                 8 * (size_t)((J + 31) / 32);
    b.cl_threads = cluster_boost_threads(J);
    // LogitBoost: one cluster of nF blocks (the slices of F, the sums, both permutations)
    const size_t ns_lb = (size_t)((J + nF - 1) / nF);
    b.lb_smem = ns_lb * 8 + std::max((size_t)P2 * 12, (size_t)J * 24) + 2 * (size_t)J + 4 +
                4 * (size_t)((J + 31) / 32);
    if (b.logit) {
        TRY(boost_cluster_fits((const void*)logitboost_cluster_kernel, o->device, nF, b.lb_smem, b.cl_threads, st, &b.cluster));
        if (!b.cluster)
            return fail(BAP_EINVAL, "LogitBoost needs a cluster of %d blocks with %zu B of shared memory each", nF, b.lb_smem);
    }
    // AdaBoost: the warp-per-feature block (form 2; by default only up to J = 2048, above which
    // the cluster's per-block scans are shorter) when its shared memory fits, else the cluster
    // (form 1) when the device can place it, else the one-block form
    b.abw_smem = warp_boost_smem(J, nF);
    {
        std::lock_guard<std::mutex> lk(g_fn_mu);
        TRY(raise_smem_limit((const void*)adaboost_kernel, o->device, g_fn[{(const void*)adaboost_kernel, o->device}]));
        FnInfo& fw = g_fn[{(const void*)adaboost_warp_kernel, o->device}];
        TRY(raise_smem_limit((const void*)adaboost_warp_kernel, o->device, fw));
        const bool want_warp = o->boost_form == 2 || (o->boost_form == 3 && J <= kWarpBoostAutoMaxJ);
        b.warp_form = !b.logit && want_warp && b.abw_smem <= fw.max_dyn_smem;
    }
    if (!b.logit && !b.warp_form && o->boost_form >= 1)
        TRY(boost_cluster_fits((const void*)adaboost_cluster_kernel, o->device, nF, b.abc_smem, b.cl_threads, st, &b.cluster));
    o->last_boost_form = b.logit ? 1 : b.warp_form ? 2 : b.cluster ? 1 : 0;
    return BAP_OK;
}

// The boosting of date m ([class]) on the J points in o->start and their labels in o->label;
// the stumps become the rule of date m.
bap_status enqueue_boost(bap_option* o, const BoostPlan& b, const bap_cmc_params* p, int m) {
    const int J = p->J, nF = o->d + 1;
    cudaStream_t st = o->stream;
    if (b.logit) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        boost_cluster_config(cfg, attr, nF, b.lb_smem, st, b.cl_threads);
        CU(cudaLaunchKernelEx(&cfg, logitboost_cluster_kernel, (const DevModel*)o->dmodel.as<DevModel>(),
                              m, J, (const double*)o->start.as<double>(),
                              (const int*)o->label.as<int>(), p->n_stumps, o->sorted_v.as<double>(),
                              o->sorted_i.as<int>(), o->max_stumps, o->n_stumps.as<int>(),
                              o->feat.as<int>(), o->thr.as<double>(), o->pol.as<int>(),
                              o->alpha.as<double>(), o->rec_len, o->rec_f.as<float>(),
                              o->rec_d.as<double>(), o->fitted.as<int>()));
    } else if (b.warp_form) {
        adaboost_warp_kernel<<<1, kWarpBoostThreads, b.abw_smem, st>>>(
            o->dmodel.as<DevModel>(), m, J, o->start.as<double>(), o->label.as<int>(),
            p->n_stumps, o->sorted_v.as<double>(), o->sorted_i.as<int>(), o->max_stumps,
            o->n_stumps.as<int>(), o->feat.as<int>(), o->thr.as<double>(), o->pol.as<int>(),
            o->alpha.as<double>(), o->rec_len, o->rec_f.as<float>(), o->rec_d.as<double>(),
            o->fitted.as<int>());
    } else if (b.cluster) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        boost_cluster_config(cfg, attr, nF, b.abc_smem, st, b.cl_threads);
        CU(cudaLaunchKernelEx(&cfg, adaboost_cluster_kernel, (const DevModel*)o->dmodel.as<DevModel>(),
                              m, J, (const double*)o->start.as<double>(),
                              (const int*)o->label.as<int>(), p->n_stumps, o->sorted_v.as<double>(),
                              o->sorted_i.as<int>(), o->max_stumps, o->n_stumps.as<int>(),
                              o->feat.as<int>(), o->thr.as<double>(), o->pol.as<int>(),
                              o->alpha.as<double>(), o->rec_len, o->rec_f.as<float>(),
                              o->rec_d.as<double>(), o->fitted.as<int>()));
    } else {
        adaboost_kernel<<<1, 1024, b.ab_smem, st>>>(
            o->dmodel.as<DevModel>(), m, J, o->start.as<double>(), o->label_y.as<double>(),
            o->label.as<int>(), p->n_stumps, o->sorted_v.as<double>(), o->sorted_i.as<int>(),
            o->err.as<double>(), o->max_stumps, o->n_stumps.as<int>(), o->feat.as<int>(),
            o->thr.as<double>(), o->pol.as<int>(), o->alpha.as<double>(), o->rec_len,
            o->rec_f.as<float>(), o->rec_d.as<double>(), o->fitted.as<int>());
    }
    ++o->launches;
    const cudaError_t eb = cudaGetLastError();
    if (eb != cudaSuccess) return fail(BAP_ECUDA, "boosting launch: %s", cudaGetErrorString(eb));
    return BAP_OK;
}

// Buffers of the boosting of J points over d+1 features.
bap_status reserve_boost(bap_option* o, int J) {
    const int nF = o->d + 1;
    TRY(o->sorted_v.reserve((size_t)nF * J * 8));
    TRY(o->sorted_i.reserve((size_t)nF * J * 4));
    TRY(o->err.reserve((size_t)nF * J * 8));
    return BAP_OK;
}

bap_status enqueue_fit_cmc(bap_option* o, const bap_cmc_params* p) {
    AllocScope scope(o->stream);
    o->launches = o->path_launches = 0;
    o->prof_used = 0;
    o->phase_used = 0;
    const bool logit = p->boost == 1;
    TRY(set_rule_cmc(o, logit ? 2 * p->n_stumps : p->n_stumps));
    o->method = 1;
    cudaStream_t st = o->stream;
    if (o->n_dates < 2) {
        o->n_items = 0;
        memset(o->pin, 0, sizeof(PinnedOut));
        CU(cudaEventRecord(o->ev0, st));
        CU(cudaEventRecord(o->ev1, st));
        return BAP_OK;
    }
    const int J = p->J;
    const int n = J;
    o->n_items = n;
    const LaunchChoice lc = tuned_launch(o->d, tune_kind(BAP_METHOD_CMC, 0), n, p->N2);
    const int chunk = choose_chunk(n, p->N2, o->unit_paths ? o->unit_paths : lc.unit);
    o->last_unit = chunk;
    const int C = (int)((p->N2 + chunk - 1) / chunk);
    const int d = o->d;
    TRY(reserve_items(o, n, (long long)n * C, 1));
    TRY(reserve_boost(o, J));
    if (p->sampler == 1) TRY(o->bridge_w.reserve((size_t)J * d * 8));
    TRY(o->diag_x.reserve((size_t)(o->n_dates + 1) * n * 8));
    TRY(o->diag_it.reserve((size_t)(o->n_dates + 1) * n * 4));
    TRY(o->diag_st.reserve((size_t)(o->n_dates + 1) * n * 4));
    CU(cudaMemsetAsync(o->diag_x.p, 0, (size_t)(o->n_dates + 1) * n * 8, st));
    CU(cudaMemsetAsync(o->diag_it.p, 0, (size_t)(o->n_dates + 1) * n * 4, st));
    CU(cudaMemsetAsync(o->diag_st.p, 0, (size_t)(o->n_dates + 1) * n * 4, st));
    CU(cudaMemsetAsync(o->done.p, 0, (size_t)n * 4, st));
    CU(cudaMemsetAsync(o->total_steps.p, 0, 8, st));
    CU(cudaMemsetAsync(o->stat_counts.p, 0, 16, st));
    BoostPlan bp;
    TRY(boost_plan(o, p, &bp));
    CU(cudaEventRecord(o->ev0, st));
    for (int m = o->n_dates - 1; m >= 1; --m) {
        const int ph_calc = phase_begin(o, PH_CALC);
        train_points_kernel<<<(J + 127) / 128, 128, 0, st>>>(
            o->dmodel.as<DevModel>(), m, make_round_keys(p->seed, P_TRAIN, (uint32_t)m), J,
            o->start.as<double>(), o->ctr_item.as<int>(),
            p->sampler == 1 ? o->bridge_w.as<double>() : nullptr, m < o->n_dates - 1 ? 1 : 0);
        ++o->launches;
        CU(cudaGetLastError());
        CU(cudaMemsetAsync(o->work.p, 0, 8, st));
        set_int_kernel<<<1, 32, 0, st>>>(o->counts.as<int>(), J);
        ++o->launches;
        PathArgs a;
        base_args(o, a, m, MODE_LABEL, false);
        a.rk = make_round_keys(p->seed, P_CMC, (uint32_t)m);
        a.N = p->N2;
        a.chunk = chunk;
        a.C = C;
        a.count = o->counts.as<int>();
        a.work = o->work.as<unsigned long long>();
        a.start = o->start.as<double>();
        a.ctr_item = o->ctr_item.as<int>();
        a.pivot = nullptr;
        a.partial = o->partial.as<double>();
        a.partial_steps = o->partial_steps.as<long long>();
        a.done = o->done.as<int>();
        a.label_y = o->label_y.as<double>();
        a.label = o->label.as<int>();
        const bap_status sl = launch_path(o, a, R_CMC, false, (long long)n * C);
        phase_end(o, ph_calc);
        TRY(sl);
        const int ph_fit = phase_begin(o, PH_FIT);
        const bap_status sb = enqueue_boost(o, bp, p, m);
        const bap_status sd = sb == BAP_OK ? record_diag(o, m, false) : BAP_OK;
        phase_end(o, ph_fit);
        TRY(sb);
        TRY(sd);
    }
    CU(cudaEventRecord(o->ev1, st));
    CU(cudaMemcpyAsync(&o->pin->fit_steps, o->total_steps.p, 8, cudaMemcpyDeviceToHost, st));
    return BAP_OK;
}

bap_status finish_fit_cmc(bap_option* o) {
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, o->ev0, o->ev1));
    o->last_fit_ms = ms;
    o->last_fit_steps = (long long)o->pin->fit_steps;
    o->last_noconv = o->last_noroot = 0;
    o->fit_launches = o->launches;
    o->fit_path_launches = o->path_launches;
    o->fit_path_ms = prof_collect(o);
    phase_collect(o);
    return BAP_OK;
}

bap_status enqueue_price(bap_option* o, int64_t n_paths, uint64_t seed) {
    AllocScope scope(o->stream);
    o->launches = o->path_launches = 0;
    o->prof_used = 0;
    o->price_n = n_paths;
    TRY(o->out_sums.reserve(3 * 8));
    TRY(o->out_steps.reserve(8));
    TRY(o->out_sums64.reserve(3 * 8));
    TRY(o->out_steps64.reserve(8));
    const RoundKeys rk = make_round_keys(seed, P_PRICE, 0);
    cudaStream_t st = o->stream;
    CU(cudaEventRecord(o->ev2, st));
    TRY(run_sums_enqueue(o, 0, MODE_SUMS, false, rk, 1, n_paths, nullptr, nullptr,
                         o->s0buf.as<double>(), o->out_sums.as<double>(), o->out_steps.as<long long>()));
    CU(cudaEventRecord(o->ev3, st));
    TRY(run_sums_enqueue(o, 0, MODE_SUMS, true, rk, 1, n_paths, nullptr, nullptr,
                         o->s0buf.as<double>(), o->out_sums64.as<double>(), o->out_steps64.as<long long>()));
    CU(cudaMemcpyAsync(o->pin->sums, o->out_sums.p, 3 * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&o->pin->steps, o->out_steps.p, 8, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(o->pin->sums64, o->out_sums64.p, 3 * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&o->pin->steps64, o->out_steps64.p, 8, cudaMemcpyDeviceToHost, st));
    return BAP_OK;
}

bap_status finish_price(bap_option* o, bap_result* res) {
    memset(res, 0, sizeof *res);
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, o->ev2, o->ev3));
    const double N = (double)o->price_n;
    const double mean = o->pin->sums[0] / N;
    double var = (o->pin->sums[1] - N * mean * mean) / (N - 1.0);
    if (var < 0) var = 0;
    res->price = mean;
    res->var = var;
    res->se = std::sqrt(var / N);
    res->ci95 = 1.96 * res->se;
    res->n_paths = o->price_n;
    res->path_steps = o->pin->steps;
    res->fp64_delta = mean - o->pin->sums64[0] / N;
    res->n_noconv = o->last_noconv;
    res->n_noroot = o->last_noroot;
    res->fit_path_steps = o->last_fit_steps;
    res->fit_ms = o->last_fit_ms;
    res->price_ms = ms;
    res->kernel_launches = o->fit_launches + o->launches;
    res->path_launches = o->fit_path_launches + o->path_launches;
    res->path_kernel_ms = o->fit_path_ms + prof_collect(o);
    for (int i = 0; i < 3; ++i) res->phase_ms[i] = o->fit_phase_ms[i];
    res->phase_ms[3] = ms;
    return BAP_OK;
}

size_t estimate_bytes(const bap_model* md, int method, const void* params, int64_t n_paths) {
    const size_t d = (size_t)md->d, nd = (size_t)md->n_dates + 1;
    size_t n = 0, slots = 0, extra = 0, rules = 0;
    if (method == BAP_METHOD_IZ) {
        const bap_iz_params* p = static_cast<const bap_iz_params*>(params);
        const size_t nb = (md->payoff == BAP_MAX_CALL && md->d > 1) ? d : 1;
        n = nb * (size_t)p->J;
        const int u = choose_chunk((long long)n, p->N1,
                                   tuned_launch(md->d, tune_kind(BAP_METHOD_IZ, p->degree), (long long)n, p->N1).unit);
        // the tail passes' slots bounded without the device's SM count
        slots = (size_t)newton_unit_slots((long long)n, p->N1, u, 1 << 20);
        extra = (size_t)(p->J + 1) * 8 + (size_t)(p->max_iter + 2) * 12;
        rules = nd * nb * (size_t)(MAXCOEF + 4) * 20;
    } else {
        const bap_cmc_params* p = static_cast<const bap_cmc_params*>(params);
        n = (size_t)p->J;
        const int u = choose_chunk((long long)n, p->N2,
                                   tuned_launch(md->d, tune_kind(BAP_METHOD_CMC, 0), (long long)n, p->N2).unit);
        slots = n * (size_t)((p->N2 + u - 1) / u);
        extra = (d + 1) * n * 20 + d * n * 8;     // sorted features, bridge state
        // stumps (feature, threshold, polarity, alpha) and the FP32 + FP64 staged records
        const size_t ms = (size_t)p->n_stumps * (p->boost == 1 ? 2 : 1);
        rules = nd * (ms * 24 + (size_t)cmc_record_len((int)d + 1, (int)ms) * 12);
    }
    const size_t items = n * (d * 8 + sizeof(ItemState) + 40) + slots * 32 + nd * n * 16;
    const size_t price_c = (size_t)((n_paths + choose_chunk(1, n_paths) - 1) / choose_chunk(1, n_paths));
    return sizeof(DevModel) + items + extra + rules + std::max(price_c, slots) * 32 + (1 << 16);
}

}  // namespace bap

// ---------------------------------------------------------------------------------------------

extern "C" {

const char* bap_last_error(void) { return error_text(); }

const char* bap_version(void) { return "bap-gb300 1.1 (sm_103a)"; }

bap_status bap_create(const bap_model* md, bap_option** out) {
    clear_error();
    return option_create(md, out);
}

bap_status bap_set_stream(bap_option* o, void* s) {
    if (!o) return fail(BAP_EINVAL, "null option");
    CU(cudaStreamSynchronize(o->stream));   // nothing of the option is pending on the old stream
    o->stream = reinterpret_cast<cudaStream_t>(s);
    return BAP_OK;
}

bap_status bap_set_profiling(bap_option* o, int on) {
    if (!o) return fail(BAP_EINVAL, "null option");
    o->profiling = on ? 1 : 0;
    o->prof_used = 0;
    return BAP_OK;
}

bap_status bap_set_launch_mode(bap_option* o, int mode) {
    if (!o) return fail(BAP_EINVAL, "null option");
    if (mode != LAUNCH_PLAIN && mode != LAUNCH_GRAPH && mode != LAUNCH_COOP)
        return fail(BAP_EINVAL, "bad launch mode");
    o->launch_mode = mode;
    return BAP_OK;
}

bap_status bap_debug_checks(bap_option* o, uint64_t* count, int* first_code) {
    if (!o || !count || !first_code) return fail(BAP_EINVAL, "null argument");
    unsigned long long h[2] = {0, 0};
    CU(cudaMemcpyAsync(h, o->check_buf.p, 16, cudaMemcpyDeviceToHost, o->stream));
    CU(cudaStreamSynchronize(o->stream));
    *count = h[0];
    *first_code = (int)h[1];
    return BAP_OK;
}

int bap_checked_build(void) {
#ifdef BAP_CHECKS
    return 1;
#else
    return 0;
#endif
}

bap_status bap_set_wait_limit(bap_option* o, uint64_t ns) {
    if (!o) return fail(BAP_EINVAL, "null option");
    o->wait_limit_ns = ns;
    return BAP_OK;
}

bap_status bap_tuned_launch(int d, int method, int degree, int64_t n_items, int64_t N,
                            int* unit_paths, int* paths_per_lane, int* from_table) {
    clear_error();
    if (!unit_paths || !paths_per_lane || d < 1 || d > MAXD || n_items < 1 || N < 1)
        return fail(BAP_EINVAL, "bad argument");
    const LaunchChoice lc = tuned_launch(d, tune_kind(method, degree), n_items, N);
    *unit_paths = choose_chunk(n_items, N, lc.unit);
    *paths_per_lane = lc.ppl;
    if (from_table) *from_table = lc.tuned ? 1 : 0;
    return BAP_OK;
}

bap_status bap_set_grid_share(bap_option* o, int share) {
    clear_error();
    if (!o || share < 1 || share > 64) return fail(BAP_EINVAL, "grid share outside 1..64");
    o->grid_share = share;
    return BAP_OK;
}

bap_status bap_set_unit_paths(bap_option* o, int paths) {
    clear_error();
    if (!o || paths < 0 || paths > 65536 || paths % 32 != 0)
        return fail(BAP_EINVAL, "unit paths must be 0 or a multiple of 32 up to 65536");
    o->unit_paths = paths;
    return BAP_OK;
}

bap_status bap_set_paths_per_lane(bap_option* o, int ppl) {
    clear_error();
    if (!o || ppl < 0 || ppl > 2) return fail(BAP_EINVAL, "paths per lane outside 0..2");
    o->ppl = ppl;
    return BAP_OK;
}

bap_status bap_set_boost_form(bap_option* o, int form) {
    if (!o) return fail(BAP_EINVAL, "null option");
    if (form < 0 || form > 3) return fail(BAP_EINVAL, "boost form outside 0..3");
    o->boost_form = form;
    return BAP_OK;
}

bap_status bap_last_boost_form(const bap_option* o, int* form) {
    if (!o || !form) return fail(BAP_EINVAL, "null argument");
    *form = o->last_boost_form;
    return BAP_OK;
}

void bap_destroy(bap_option* o) { option_destroy(o); }

bap_status bap_fit_boundary(bap_option* o, const bap_iz_params* p) {
    clear_error();
    if (!o) return fail(BAP_EINVAL, "null option");
    TRY(validate_iz(o->d, p));
    TRY(enqueue_fit_iz(o, p));
    CU(cudaStreamSynchronize(o->stream));
    return finish_fit_iz(o);
}

bap_status bap_fit_classifier(bap_option* o, const bap_cmc_params* p) {
    clear_error();
    if (!o) return fail(BAP_EINVAL, "null option");
    TRY(validate_cmc(o, p));
    TRY(enqueue_fit_cmc(o, p));
    CU(cudaStreamSynchronize(o->stream));
    return finish_fit_cmc(o);
}

bap_status bap_price(bap_option* o, int64_t n_paths, uint64_t seed, bap_result* res) {
    clear_error();
    if (!res) return fail(BAP_EINVAL, "null argument");
    TRY(validate_price(o, n_paths));
    TRY(enqueue_price(o, n_paths, seed));
    CU(cudaStreamSynchronize(o->stream));
    return finish_price(o, res);
}

namespace {
bap_status debug_continuation_impl(bap_option* o, int m, int purpose, uint64_t seed, int n_items,
                                   const int* item_ids, const int* pivots, const double* starts,
                                   int64_t N, double* sums, int64_t* steps, bool fp64) {
    if (!o || !item_ids || !starts || !sums || !steps) return fail(BAP_EINVAL, "null argument");
    if (m < 1 || m >= o->n_dates) return fail(BAP_EINVAL, "m=%d outside 1..n_dates-1", m);
    if (n_items < 1 || N < 1 || N > (1LL << 31)) return fail(BAP_EINVAL, "bad n_items or N");
    if (purpose < 1 || purpose > 4) return fail(BAP_EINVAL, "bad purpose");
    const int d = o->d;
    AllocScope scope(o->stream);
    for (int i = 0; i < n_items; ++i) {
        for (int q = 0; q < d; ++q)
            if (!(starts[(size_t)i * d + q] > 0)) return fail(BAP_EINVAL, "start points must be positive");
        if (pivots && (pivots[i] < -1 || pivots[i] >= d)) return fail(BAP_EINVAL, "bad pivot");
    }
    DevBuf ds, di, dp;
    TRY(ds.reserve((size_t)n_items * d * 8));
    TRY(di.reserve((size_t)n_items * 4));
    if (pivots) TRY(dp.reserve((size_t)n_items * 4));
    CU(cudaMemcpyAsync(ds.p, starts, (size_t)n_items * d * 8, cudaMemcpyHostToDevice, o->stream));
    CU(cudaMemcpyAsync(di.p, item_ids, (size_t)n_items * 4, cudaMemcpyHostToDevice, o->stream));
    if (pivots) CU(cudaMemcpyAsync(dp.p, pivots, (size_t)n_items * 4, cudaMemcpyHostToDevice, o->stream));
    std::vector<long long> st(n_items);
    TRY(run_sums(o, m, MODE_SUMS, fp64, make_round_keys(seed, (uint32_t)purpose, (uint32_t)m), n_items, N,
                 di.as<int>(), pivots ? dp.as<int>() : nullptr, ds.as<double>(), sums, st.data()));
    for (int i = 0; i < n_items; ++i) steps[i] = st[i];
    return BAP_OK;
}
}  // namespace

bap_status bap_debug_continuation(bap_option* o, int m, int purpose, uint64_t seed, int n_items,
                                  const int* item_ids, const int* pivots, const double* starts,
                                  int64_t N, double* sums, int64_t* steps) {
    clear_error();
    return debug_continuation_impl(o, m, purpose, seed, n_items, item_ids, pivots, starts, N, sums,
                                   steps, false);
}

bap_status bap_debug_continuation_fp64(bap_option* o, int m, int purpose, uint64_t seed,
                                       int n_items, const int* item_ids, const int* pivots,
                                       const double* starts, int64_t N, double* sums,
                                       int64_t* steps) {
    clear_error();
    return debug_continuation_impl(o, m, purpose, seed, n_items, item_ids, pivots, starts, N, sums,
                                   steps, true);
}

bap_status bap_debug_paths(bap_option* o, int m, int purpose, uint64_t seed, int item_id,
                           const double* start, int64_t N, int* tau, double* disc_phi) {
    clear_error();
    if (!o || !start || !tau || !disc_phi) return fail(BAP_EINVAL, "null argument");
    if (m < 0 || m >= o->n_dates) return fail(BAP_EINVAL, "bad m");
    if (N < 1 || N > (1LL << 26)) return fail(BAP_EINVAL, "N outside 1..2^26");
    const int d = o->d;
    AllocScope scope(o->stream);
    DevBuf ds, di;
    TRY(ds.reserve((size_t)d * 8));
    TRY(di.reserve(4));
    TRY(o->trace_tau.reserve((size_t)N * 4));
    TRY(o->trace_phi.reserve((size_t)N * 8));
    CU(cudaMemcpyAsync(ds.p, start, (size_t)d * 8, cudaMemcpyHostToDevice, o->stream));
    CU(cudaMemcpyAsync(di.p, &item_id, 4, cudaMemcpyHostToDevice, o->stream));
    double sums[3];
    long long steps;
    TRY(run_sums(o, m, MODE_TRACE, false, make_round_keys(seed, (uint32_t)purpose, (uint32_t)m), 1, N,
                 di.as<int>(), nullptr, ds.as<double>(), sums, &steps));
    CU(cudaMemcpy(tau, o->trace_tau.p, (size_t)N * 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(disc_phi, o->trace_phi.p, (size_t)N * 8, cudaMemcpyDeviceToHost));
    return BAP_OK;
}

bap_status bap_debug_newton(bap_option* o, const bap_iz_params* p, int m, int n_items,
                            const int* item_ids, const int* pivots, const double* starts,
                            double* x, int* iters, int* status, double* lo, double* hi,
                            int64_t* path_steps) {
    clear_error();
    if (!o || !p || !item_ids || !pivots || !starts || !x || !iters || !status)
        return fail(BAP_EINVAL, "null argument");
    TRY(validate_iz(o->d, p));
    if (m < 1 || m >= o->n_dates) return fail(BAP_EINVAL, "m=%d outside 1..n_dates-1", m);
    if (n_items < 1 || n_items > (1 << 24)) return fail(BAP_EINVAL, "n_items outside 1..2^24");
    if (o->rule_kind == R_CMC) return fail(BAP_ESTATE, "the option holds a CMC rule, not boundaries");
    const int d = o->d;
    for (int i = 0; i < n_items; ++i) {
        if (pivots[i] < 0 || pivots[i] >= d) return fail(BAP_EINVAL, "pivot outside 0..d-1");
        for (int q = 0; q < d; ++q)
            if (q != pivots[i] && !(starts[(size_t)i * d + q] > 0))
                return fail(BAP_EINVAL, "start points must be positive");
    }
    AllocScope scope(o->stream);
    cudaStream_t st = o->stream;
    const int n_bnd = (o->payoff == BAP_MAX_CALL && d > 1) ? d : 1;
    const LaunchChoice lc = tuned_launch(d, tune_kind(BAP_METHOD_IZ, o->degree), n_items, p->N1);
    const int chunk = choose_chunk(n_items, p->N1, o->unit_paths ? o->unit_paths : lc.unit);
    const int C = (int)((p->N1 + chunk - 1) / chunk);
    o->ppl_fit = lc.ppl;
    TRY(reserve_items(o, n_items, newton_unit_slots(n_items, p->N1, chunk, o->sm_count), p->max_iter));
    DevBuf ds, dp, di, dl;
    TRY(ds.reserve((size_t)n_items * d * 8));
    TRY(dp.reserve((size_t)n_items * 4));
    TRY(di.reserve((size_t)n_items * 4));
    TRY(dl.reserve((size_t)n_items * 4));
    CU(cudaMemcpyAsync(ds.p, starts, (size_t)n_items * d * 8, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(dp.p, pivots, (size_t)n_items * 4, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(di.p, item_ids, (size_t)n_items * 4, cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(o->done.p, 0, (size_t)n_items * 4, st));
    CU(cudaMemsetAsync(o->total_steps.p, 0, 8, st));
    CU(cudaMemsetAsync(o->stat_counts.p, 0, 16, st));
    CU(cudaMemsetAsync(o->counts.p, 0, (size_t)(p->max_iter + 2) * 4, st));
    CU(cudaMemsetAsync(o->work.p, 0, (size_t)(p->max_iter + 2) * 8, st));
    const bool warm = p->warm_start && o->rule_kind == R_IZ;
    newton_items_setup_kernel<<<(n_items + 127) / 128, 128, 0, st>>>(
        o->dmodel.as<DevModel>(), m, n_items, n_bnd, ds.as<double>(), dp.as<int>(), di.as<int>(),
        o->start.as<double>(), o->state.as<ItemState>(), o->pivot.as<int>(), o->ctr_item.as<int>(),
        dl.as<int>(), warm ? o->coef64.as<double>() : nullptr, o->n_coef, o->degree,
        o->fitted.as<int>(), warm ? 1 : 0, o->l0f.as<float>());
    newton_items_list_kernel<<<1, 32, 0, st>>>(dl.as<int>(), n_items, o->active0.as<int>(), o->counts.as<int>());
    CU(cudaGetLastError());
    // the fit's own Newton launches, on these items (the option's fit diagnostics stay as they are)
    const int saved_n = o->n_items;
    o->n_items = n_items;
    bap_status sn = BAP_OK;
    if (o->launch_mode == LAUNCH_COOP) {
        sn = enqueue_newton_coop(o, p, m, chunk, C);
    } else {
        for (int it = 0; it < p->max_iter && sn == BAP_OK; ++it)
            sn = enqueue_newton_pass(o, p, m, it, chunk, C);
    }
    o->n_items = saved_n;
    TRY(sn);
    std::vector<ItemState> hs(n_items);
    int flags[4] = {0, 0, 0, 0};
    unsigned long long steps = 0;
    CU(cudaMemcpyAsync(hs.data(), o->state.p, (size_t)n_items * sizeof(ItemState), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(flags, o->stat_counts.p, 16, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&steps, o->total_steps.p, 8, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (flags[3] != 0) return fail(BAP_ECUDA, "Newton loop: a grid barrier of the cooperative launch timed out");
    for (int i = 0; i < n_items; ++i) {
        x[i] = hs[i].x;
        iters[i] = hs[i].iters;
        status[i] = hs[i].status;
        if (lo) lo[i] = hs[i].lo;
        if (hi) hi[i] = hs[i].hi;
    }
    if (path_steps) *path_steps = (int64_t)steps;
    return BAP_OK;
}

bap_status bap_debug_ls_fit(bap_option* o, int degree, int J, const double* starts,
                            const double* x, const int* status, double* coef) {
    clear_error();
    if (!o || !starts || !x || !status || !coef) return fail(BAP_EINVAL, "null argument");
    const int d = o->d, s = d - 1;
    if (s == 0) degree = 0;
    if (degree < 0 || degree > 3 || (degree == 3 && d > MAXD_CUBIC)) return fail(BAP_EINVAL, "bad degree");
    if (J < 1 || J > 8192) return fail(BAP_EINVAL, "J outside 1..8192");
    const int n_bnd = (o->payoff == BAP_MAX_CALL && d > 1) ? d : 1;
    const int n = n_bnd * J;
    const int P = n_basis(s, degree);
    for (int i = 0; i < n; ++i)
        if (status[i] < 0 || status[i] > 2) return fail(BAP_EINVAL, "status outside 0..2");
    AllocScope scope(o->stream);
    cudaStream_t st = o->stream;
    std::vector<ItemState> hs(n);
    for (int i = 0; i < n; ++i) {
        memset(&hs[i], 0, sizeof(ItemState));
        hs[i].x = x[i];
        hs[i].status = status[i];
    }
    DevBuf ds, dst, dc, dcf, dcd, dfit;
    TRY(ds.reserve((size_t)n * d * 8));
    TRY(dst.reserve((size_t)n * sizeof(ItemState)));
    TRY(dc.reserve((size_t)n_bnd * P * 8));
    TRY(dcf.reserve((size_t)n_bnd * iz_stride(d, degree) * 4));
    TRY(dcd.reserve((size_t)n_bnd * iz_stride(d, degree) * 8));
    TRY(dfit.reserve(16));
    CU(cudaMemcpyAsync(ds.p, starts, (size_t)n * d * 8, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(dst.p, hs.data(), (size_t)n * sizeof(ItemState), cudaMemcpyHostToDevice, st));
    ls_fit_kernel<<<n_bnd, kLsThreads, 0, st>>>(o->dmodel.as<DevModel>(), 0, J, n_bnd, degree, P,
                                                ds.as<double>(), dst.as<ItemState>(), dc.as<double>(),
                                                dcf.as<float>(), dcd.as<double>(), dfit.as<int>());
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(coef, dc.p, (size_t)n_bnd * P * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return BAP_OK;
}

bap_status bap_debug_boost(bap_option* o, const bap_cmc_params* p, int m, const double* X,
                           const int* labels, int* n_stumps, double* stumps) {
    clear_error();
    if (!o || !p || !X || !labels || !n_stumps || !stumps) return fail(BAP_EINVAL, "null argument");
    TRY(validate_cmc(o, p));
    if (m < 1 || m >= o->n_dates) return fail(BAP_EINVAL, "m=%d outside 1..n_dates-1", m);
    const int d = o->d, J = p->J;
    for (int j = 0; j < J; ++j) {
        if (labels[j] != 1 && labels[j] != -1) return fail(BAP_EINVAL, "labels must be +1 or -1");
        for (int q = 0; q < d; ++q)
            if (!(X[(size_t)j * d + q] > 0)) return fail(BAP_EINVAL, "points must be positive");
    }
    AllocScope scope(o->stream);
    cudaStream_t st = o->stream;
    const int ms = p->boost == 1 ? 2 * p->n_stumps : p->n_stumps;
    if (o->rule_kind != R_CMC || o->max_stumps != ms) TRY(set_rule_cmc(o, ms));
    TRY(o->start.reserve((size_t)J * d * 8));
    TRY(o->label.reserve((size_t)J * 4));
    TRY(o->label_y.reserve((size_t)J * 8));
    TRY(reserve_boost(o, J));
    CU(cudaMemcpyAsync(o->start.p, X, (size_t)J * d * 8, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(o->label.p, labels, (size_t)J * 4, cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(o->label_y.p, 0, (size_t)J * 8, st));
    BoostPlan bp;
    TRY(boost_plan(o, p, &bp));
    TRY(enqueue_boost(o, bp, p, m));
    const size_t base = (size_t)m * ms;
    std::vector<int> f(ms), pl(ms);
    std::vector<double> th(ms), al(ms);
    int cnt = 0;
    CU(cudaMemcpyAsync(&cnt, o->n_stumps.as<int>() + m, 4, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(f.data(), o->feat.as<int>() + base, ms * 4, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(pl.data(), o->pol.as<int>() + base, ms * 4, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(th.data(), o->thr.as<double>() + base, ms * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(al.data(), o->alpha.as<double>() + base, ms * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    *n_stumps = cnt;
    for (int i = 0; i < ms; ++i) {
        stumps[4 * i + 0] = f[i];
        stumps[4 * i + 1] = th[i];
        stumps[4 * i + 2] = pl[i];
        stumps[4 * i + 3] = al[i];
    }
    return BAP_OK;
}

bap_status bap_debug_rng(uint64_t seed, int purpose, int m, uint32_t w1, uint32_t step, int d,
                         int64_t count, uint32_t* words, double* z) {
    clear_error();
    if (d < 1 || d > 16 || count < 1 || count > (1LL << 26)) return fail(BAP_EINVAL, "bad d or count");
    int dev;
    if (!has_device(&dev)) return fail(BAP_ECUDA, "no CUDA device");
    const int nc = (d + 3) / 4;
    AllocScope scope(nullptr);
    DevBuf dw, dz;
    if (words) TRY(dw.reserve((size_t)count * nc * 16));
    if (z) TRY(dz.reserve((size_t)count * d * 8));
    rng_debug_kernel<<<(unsigned)((count + 255) / 256), 256>>>(
        make_round_keys(seed, (uint32_t)purpose, (uint32_t)m), w1, step, d, count,
        words ? dw.as<uint32_t>() : nullptr, z ? dz.as<double>() : nullptr);
    CU(cudaGetLastError());
    if (words) CU(cudaMemcpy(words, dw.p, (size_t)count * nc * 16, cudaMemcpyDeviceToHost));
    if (z) CU(cudaMemcpy(z, dz.p, (size_t)count * d * 8, cudaMemcpyDeviceToHost));
    return BAP_OK;
}

bap_status bap_fit_points(const bap_option* o, int m, int* n_items, double* x, int* iters, int* status) {
    clear_error();
    if (!o || !n_items) return fail(BAP_EINVAL, "null argument");
    if (o->method < 0) return fail(BAP_ESTATE, "no fit yet");
    if (m < 1 || m >= o->n_dates) return fail(BAP_EINVAL, "bad m");
    const int n = o->n_items;
    const int cap = *n_items;
    *n_items = n;
    if (!x && !iters && !status) return BAP_OK;
    const int k = std::min(cap, n);
    if (k <= 0) return BAP_OK;
    CU(cudaStreamSynchronize(o->stream));
    if (x) CU(cudaMemcpy(x, o->diag_x.as<double>() + (size_t)m * n, (size_t)k * 8, cudaMemcpyDeviceToHost));
    if (iters) CU(cudaMemcpy(iters, o->diag_it.as<int>() + (size_t)m * n, (size_t)k * 4, cudaMemcpyDeviceToHost));
    if (status) CU(cudaMemcpy(status, o->diag_st.as<int>() + (size_t)m * n, (size_t)k * 4, cudaMemcpyDeviceToHost));
    return BAP_OK;
}

bap_status bap_export_rules(const bap_option* o, double* buf, size_t* len) {
    clear_error();
    if (!o || !len) return fail(BAP_EINVAL, "null argument");
    const int nd = o->n_dates + 1;
    const int kind = o->rule_kind;
    size_t need = 6 + nd;
    if (kind == R_IZ) need += (size_t)nd * o->n_bnd * o->n_coef;
    if (kind == R_CMC) need += (size_t)nd * o->max_stumps * 4 + nd;
    if (!buf) { *len = need; return BAP_OK; }
    std::vector<double> out(need, 0.0);
    out[0] = kind;
    out[1] = o->n_dates;
    out[2] = o->n_bnd;
    out[3] = o->degree;
    out[4] = o->n_coef;
    out[5] = o->max_stumps;
    std::vector<int> fit(nd);
    CU(cudaStreamSynchronize(o->stream));
    CU(cudaMemcpy(fit.data(), o->fitted.p, nd * 4, cudaMemcpyDeviceToHost));
    for (int k = 0; k < nd; ++k) out[6 + k] = fit[k];
    size_t off = 6 + nd;
    if (kind == R_IZ) {
        CU(cudaMemcpy(out.data() + off, o->coef64.p, (size_t)nd * o->n_bnd * o->n_coef * 8, cudaMemcpyDeviceToHost));
    } else if (kind == R_CMC) {
        const size_t ns = (size_t)nd * o->max_stumps;
        std::vector<int> f(ns), pl(ns), nst(nd);
        std::vector<double> th(ns), al(ns);
        CU(cudaMemcpy(f.data(), o->feat.p, ns * 4, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(pl.data(), o->pol.p, ns * 4, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(th.data(), o->thr.p, ns * 8, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(al.data(), o->alpha.p, ns * 8, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(nst.data(), o->n_stumps.p, nd * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < ns; ++i) {
            out[off + 4 * i + 0] = f[i];
            out[off + 4 * i + 1] = th[i];
            out[off + 4 * i + 2] = pl[i];
            out[off + 4 * i + 3] = al[i];
        }
        for (int k = 0; k < nd; ++k) out[off + 4 * ns + k] = nst[k];
    }
    memcpy(buf, out.data(), std::min(*len, need) * 8);
    *len = need;
    return BAP_OK;
}

bap_status bap_import_rules(bap_option* o, const double* buf, size_t len) {
    clear_error();
    if (!o || !buf || len < 6) return fail(BAP_EINVAL, "null or short buffer");
    AllocScope scope(o->stream);
    const int kind = (int)buf[0];
    const int nd = o->n_dates + 1;
    if ((int)buf[1] != o->n_dates) return fail(BAP_EINVAL, "n_dates mismatch");
    if (len < (size_t)(6 + nd)) return fail(BAP_EINVAL, "short buffer");
    std::vector<int> fit(nd);
    for (int k = 0; k < nd; ++k) fit[k] = buf[6 + k] != 0.0;
    const size_t off = 6 + nd;
    if (kind == R_NONE) {
        o->rule_kind = R_NONE;
        CU(cudaMemsetAsync(o->fitted.p, 0, nd * 4, o->stream));
        CU(cudaStreamSynchronize(o->stream));
        return BAP_OK;
    }
    if (kind == R_IZ) {
        const int degree = (int)buf[3];
        if (degree < 0 || degree > 3 || (degree == 3 && o->d > MAXD_CUBIC))
            return fail(BAP_EINVAL, "bad degree");
        TRY(set_rule_iz(o, degree));
        if ((int)buf[2] != o->n_bnd || (int)buf[4] != o->n_coef) return fail(BAP_EINVAL, "boundary shape mismatch");
        const size_t nc = (size_t)nd * o->n_bnd * o->n_coef;
        if (len < off + nc) return fail(BAP_EINVAL, "short buffer");
        for (size_t i = 0; i < nc; ++i)
            if (!std::isfinite(buf[off + i])) return fail(BAP_EINVAL, "non-finite boundary coefficient");
        CU(cudaMemcpyAsync(o->coef64.p, buf + off, nc * 8, cudaMemcpyHostToDevice, o->stream));
        stage_iz_kernel<<<(nd * o->n_bnd + 127) / 128, 128, 0, o->stream>>>(
            o->coef64.as<double>(), o->n_dates, o->n_bnd, o->n_coef, o->d - 1, o->degree, o->K,
            o->coef_f.as<float>(), o->coef_d.as<double>());
        CU(cudaGetLastError());
    } else if (kind == R_CMC) {
        const int ms = (int)buf[5];
        if (ms < 1 || ms > BAP_MAX_STUMPS) return fail(BAP_EINVAL, "bad max_stumps");
        TRY(set_rule_cmc(o, ms));
        const size_t ns = (size_t)nd * ms;
        if (len < off + 4 * ns + nd) return fail(BAP_EINVAL, "short buffer");
        std::vector<int> f(ns), pl(ns), nst(nd);
        std::vector<double> th(ns), al(ns);
        for (size_t i = 0; i < ns; ++i) {
            f[i] = (int)buf[off + 4 * i];
            th[i] = buf[off + 4 * i + 1];
            pl[i] = (int)buf[off + 4 * i + 2];
            al[i] = buf[off + 4 * i + 3];
            if (f[i] < 0 || f[i] > o->d || (pl[i] != 1 && pl[i] != -1 && al[i] != 0.0) ||
                std::isnan(th[i]) || !std::isfinite(al[i]))
                return fail(BAP_EINVAL, "bad stump");
        }
        for (int k = 0; k < nd; ++k) {
            nst[k] = (int)buf[off + 4 * ns + k];
            if (nst[k] < 0 || nst[k] > ms) return fail(BAP_EINVAL, "bad stump count");
        }
        CU(cudaMemcpyAsync(o->feat.p, f.data(), ns * 4, cudaMemcpyHostToDevice, o->stream));
        CU(cudaMemcpyAsync(o->pol.p, pl.data(), ns * 4, cudaMemcpyHostToDevice, o->stream));
        CU(cudaMemcpyAsync(o->thr.p, th.data(), ns * 8, cudaMemcpyHostToDevice, o->stream));
        CU(cudaMemcpyAsync(o->alpha.p, al.data(), ns * 8, cudaMemcpyHostToDevice, o->stream));
        CU(cudaMemcpyAsync(o->n_stumps.p, nst.data(), nd * 4, cudaMemcpyHostToDevice, o->stream));
        stage_cmc_kernel<<<(nd + 31) / 32, 32, 0, o->stream>>>(
            o->n_dates, o->d + 1, ms, o->n_stumps.as<int>(), o->feat.as<int>(), o->thr.as<double>(),
            o->pol.as<int>(), o->alpha.as<double>(), o->rec_len, o->rec_f.as<float>(), o->rec_d.as<double>());
        CU(cudaGetLastError());
    } else {
        return fail(BAP_EINVAL, "bad rule kind %d", kind);
    }
    CU(cudaMemcpyAsync(o->fitted.p, fit.data(), nd * 4, cudaMemcpyHostToDevice, o->stream));
    CU(cudaStreamSynchronize(o->stream));
    return BAP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Continuation sums for callers that cannot allocate device memory.
//
// The scratch of the path kernel (per-unit partial sums, per-item unit counters, the work
// counter, the item count and the step total) lives in one fixed array in this library's device
// image instead of in buffers from cudaMalloc.  Every GPU that loads the library holds the array
// until the process exits.  Host code never names the array as an address: every call looks its
// address up with cudaGetSymbolAddress, with the option's device current (the first lookup on a
// device loads the library's device image there if that has not happened yet).  All calls
// share the array and it keeps the last call's contents, so the call clears what must start at
// zero; calls whose work overlaps on the GPU race on it.

#define BAP_STATIC_SCRATCH_BYTES (4u << 20)

static __device__ __align__(256) unsigned char bap_static_scratch[BAP_STATIC_SCRATCH_BYTES];

namespace {

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Header of the array: [0] work counter (u64), [8] step total (u64), [16] item count (int).
// Besides clearing, this kernel checks the caller's inputs on the device: an item whose pivot is
// outside -1..d-1 or whose start point has a coordinate that is not positive is marked bad, and
// the path kernel gets a copy of the pivots with such pivots replaced by -1, so that no pivot
// ever indexes outside the item's start point.
__global__ void static_scratch_clear_kernel(unsigned char* base, int n_items, int d, size_t done_off,
                                            size_t piv_off, size_t bad_off, const int* pivots,
                                            const double* starts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *reinterpret_cast<unsigned long long*>(base) = 0ULL;
        *reinterpret_cast<unsigned long long*>(base + 8) = 0ULL;
        *reinterpret_cast<int*>(base + 16) = n_items;
    }
    int* done = reinterpret_cast<int*>(base + done_off);
    int* piv = reinterpret_cast<int*>(base + piv_off);
    int* bad = reinterpret_cast<int*>(base + bad_off);
    for (int k = i; k < n_items; k += gridDim.x * blockDim.x) {
        done[k] = 0;
        int b = 0;
        int p = pivots ? pivots[k] : -1;
        if (p < -1 || p >= d) { b = 1; p = -1; }
        for (int q = 0; q < d; ++q)
            if (!(starts[(size_t)k * d + q] > 0.0)) b = 1;   // also catches NaN
        piv[k] = p;
        bad[k] = b;
    }
}

// Items marked bad get NaN sums and -1 steps (their paths ran on the clamped pivot; no access
// left the caller's buffers).
__global__ void static_mark_bad_kernel(const int* bad, int n_items, double* sums, long long* steps) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_items; k += gridDim.x * blockDim.x) {
        if (bad[k]) {
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
            sums[3 * (size_t)k + 0] = nan;
            sums[3 * (size_t)k + 1] = nan;
            sums[3 * (size_t)k + 2] = nan;
            steps[k] = -1;
        }
    }
}

}  // namespace

extern "C" bap_status bap_continuation_static(bap_option* o, int m, int purpose, uint64_t seed,
                                              int n_items, const int* d_item_ids,
                                              const int* d_pivots, const double* d_starts,
                                              int64_t N, double* d_sums, int64_t* d_steps) {
    g_err.clear();
    if (!o || !d_item_ids || !d_starts || !d_sums || !d_steps) return fail(BAP_EINVAL, "null argument");
    if (m < 1 || m >= o->n_dates) return fail(BAP_EINVAL, "m=%d outside 1..n_dates-1", m);
    if (n_items < 1 || N < 1 || N > (1LL << 31)) return fail(BAP_EINVAL, "bad n_items or N");
    if (purpose < 1 || purpose > 4) return fail(BAP_EINVAL, "bad purpose");
    const int chunk = choose_chunk(n_items, N);
    const long long C = (N + chunk - 1) / chunk;
    const long long units = (long long)n_items * C;
    const size_t done_off = 256;
    const size_t piv_off = done_off + align256((size_t)n_items * 4);
    const size_t bad_off = piv_off + align256((size_t)n_items * 4);
    const size_t steps_off = bad_off + align256((size_t)n_items * 4);
    const size_t partial_off = steps_off + align256((size_t)units * 8);
    const size_t need = partial_off + (size_t)units * 24;
    if (need > BAP_STATIC_SCRATCH_BYTES)
        return fail(BAP_EINVAL,
                    "n_items=%d with N=%lld needs %zu bytes of scratch; the static scratch holds %u "
                    "bytes (use bap_debug_continuation, which allocates)",
                    n_items, (long long)N, need, (unsigned)BAP_STATIC_SCRATCH_BYTES);
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != o->device) return fail(BAP_EINVAL, "the option's device %d is not current (%d)", o->device, dev);
    // The array's device address, looked up on every call (cheap next to the kernels): after a
    // device reset the image may be loaded at another address.
    unsigned char* base = nullptr;
    {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, bap_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(BAP_ECUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
        base = static_cast<unsigned char*>(p);
    }
    const int clear_blocks = std::max(1, std::min(1024, (n_items + 255) / 256));
    static_scratch_clear_kernel<<<clear_blocks, 256, 0, o->stream>>>(
        base, n_items, o->d, done_off, piv_off, bad_off, d_pivots, d_starts);
    ++o->launches;
    CU(cudaGetLastError());

    PathArgs a;
    base_args(o, a, m, MODE_SUMS, false);
    a.n_items = n_items;
    a.rk = make_round_keys(seed, (uint32_t)purpose, (uint32_t)m);
    a.N = N;
    a.chunk = chunk;
    a.C = (int)C;
    a.count = reinterpret_cast<int*>(base + 16);
    a.work = reinterpret_cast<unsigned long long*>(base);
    a.total_steps = reinterpret_cast<unsigned long long*>(base + 8);
    a.start = const_cast<double*>(d_starts);
    a.ctr_item = d_item_ids;
    a.pivot = d_pivots ? reinterpret_cast<const int*>(base + piv_off) : nullptr;
    a.done = reinterpret_cast<int*>(base + done_off);
    a.partial_steps = reinterpret_cast<long long*>(base + steps_off);
    a.partial = reinterpret_cast<double*>(base + partial_off);
    a.out_sums = d_sums;
    a.out_steps = reinterpret_cast<long long*>(d_steps);
    TRY(launch_path(o, a, o->rule_kind, false, units, /*no_events=*/true));
    static_mark_bad_kernel<<<clear_blocks, 256, 0, o->stream>>>(
        reinterpret_cast<const int*>(base + bad_off), n_items, d_sums, reinterpret_cast<long long*>(d_steps));
    ++o->launches;
    CU(cudaGetLastError());
    return BAP_OK;
}
