// bap_host.cuh -- host-side state of an option and the asynchronous building blocks that the C
// ABI (bap_api.cu) and the serving loop (bap_server.cu) share.  Private to the library.
#pragma once

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bap_fit.cuh"
#include "bap_path.cuh"

namespace bap {

// Thread-local message of the last failure (bap_last_error).
bap_status fail(bap_status st, const char* fmt, ...);
void clear_error();
const char* error_text();

#define CU(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return ::bap::fail(e_ == cudaErrorMemoryAllocation ? BAP_ENOMEM : BAP_ECUDA,     \
                               "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,    \
                               __LINE__);                                                    \
    } while (0)

#define TRY(expr)                          \
    do {                                   \
        bap_status s_ = (expr);            \
        if (s_ != BAP_OK) return s_;       \
    } while (0)

// Stream on which DevBuf allocations of the calling thread are ordered (set by AllocScope at
// every entry point that may allocate; the legacy default stream otherwise).
cudaStream_t& alloc_stream();

struct AllocScope {
    cudaStream_t prev;
    explicit AllocScope(cudaStream_t s) : prev(alloc_stream()) { alloc_stream() = s; }
    ~AllocScope() { alloc_stream() = prev; }
};

// A device buffer that grows on demand.  Memory comes from the device's stream-ordered pool
// (cudaMallocAsync / cudaFreeAsync on the allocating stream): unlike cudaMalloc and cudaFree,
// these never wait for the whole device, so options in flight on other streams keep running.
struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;     // stream of the allocation
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(s); }
    void release(cudaStream_t on) {
        if (p) cudaFreeAsync(p, on);
        p = nullptr;
        n = 0;
    }
    bap_status reserve(size_t bytes) {
        if (bytes <= n) return BAP_OK;
        cudaStream_t st = alloc_stream();
        release(st);
        const size_t want = bytes < 256 ? 256 : bytes;
        cudaError_t e = cudaMallocAsync(&p, want, st);
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(BAP_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
        }
        n = want;
        s = st;
        return BAP_OK;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Results an enqueued fit or pricing leaves in page-locked host memory.
struct PinnedOut {
    unsigned long long fit_steps;
    int counts[4];                // [0] points without convergence, [1] points without a root
    double sums[3];               // pricing, FP32 paths
    long long steps;
    double sums64[3];             // pricing, FP64 paths
    long long steps64;
};

// Launch form of the I&Z Newton passes: one launch per pass (max_iter per date), one graph for
// the whole fit (conditional while node per date), or one cooperative launch per date.
enum LaunchMode : int { LAUNCH_PLAIN = 0, LAUNCH_GRAPH = 1, LAUNCH_COOP = 2 };

// Page-locked result blocks come from a slab that is never freed (cudaFreeHost would wait for
// the whole device).
PinnedOut* pinned_get();
void pinned_put(PinnedOut* p);

}  // namespace bap

struct bap_option {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    // model (host copies)
    int d = 0, n_dates = 0, payoff = 0;
    double r = 0, K = 0, T = 0;
    bap::DevModel hm{};           // host copy after device set-up
    bap::DevBuf dmodel, s0buf;
    // rule
    int rule_kind = bap::R_NONE;
    int n_bnd = 1, degree = 0, n_coef = 1;
    int max_stumps = 0, rec_len = 0;
    bap::DevBuf fitted;           // int[n_dates+1]
    bap::DevBuf coef64, coef_f, coef_d;
    bap::DevBuf n_stumps, feat, thr, pol, alpha, rec_f, rec_d;
    // fit state and scratch
    int method = -1;              // last fit: 0 I&Z, 1 CMC
    int n_items = 0;
    bap::DevBuf start, state, pivot, ctr_item, active0, active1, counts, work, partial,
        partial_steps, done, total_steps, l0f, korobov_a, merit, label_y, label, sorted_v, sorted_i,
        err, out_sums, out_steps, out_sums64, out_steps64, trace_tau, trace_phi, diag_x, diag_it,
        diag_st, stat_counts, one, iterstate, bridge_w, check_buf;
    int last_noconv = 0, last_noroot = 0;
    long long last_fit_steps = 0;
    double last_fit_ms = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
    bap::PinnedOut* pin = nullptr;
    int64_t price_n = 0;
    // launch accounting and optional per-launch timing of the path kernel
    long long launches = 0, path_launches = 0;
    long long fit_launches = 0, fit_path_launches = 0;
    double fit_path_ms = 0;
    int profiling = 0;
    int capturing = 0;
    std::vector<cudaEvent_t> prof_ev;
    size_t prof_used = 0;
    // per-phase device time of the last fit (profiling on): [0] glp, [1] calc, [2] reg / class
    struct PhaseMark { int phase; cudaEvent_t a, b; };
    std::vector<PhaseMark> phase_ev;
    size_t phase_used = 0;
    double fit_phase_ms[3] = {0, 0, 0};
    // graph of the I&Z fit (Newton loops as conditional while nodes)
    int launch_mode = bap::LAUNCH_GRAPH;
    int grid_share = 1;           // cooperative launches use at most 1/grid_share of the device
    unsigned long long wait_limit_ns = 0;   // grid-barrier wait bound; 0: automatic
    int boost_form = 3;           // CMC boosting: 3 by J, 2 warp per feature, 1 cluster, 0 one block
    int ppl = 0;                  // path slots per lane of the FP32 quadratic I&Z kernels (0: tuned)
    int ppl_fit = 1;              // the tuned choice for the current fit's Newton launches
    int unit_paths = 0;           // paths per warp unit of the fits' path launches (0: tuned)
    int last_unit = 0;            // paths per unit the last fit ran with
    int last_boost_form = 0;      // form the last CMC fit ran
    cudaGraphExec_t graph_exec = nullptr;
    bap_iz_params graph_params{};
    int graph_chunk = 0;          // unit size the graph was built with
    int graph_failed = 0;
    int last_graph = 0;

    template <typename F> void for_each_buf(F f) {
        bap::DevBuf* all[] = {&dmodel, &s0buf, &fitted, &coef64, &coef_f, &coef_d, &n_stumps,
                              &feat, &thr, &pol, &alpha, &rec_f, &rec_d, &start, &state, &pivot,
                              &ctr_item, &active0, &active1, &counts, &work, &partial,
                              &partial_steps, &done, &total_steps, &l0f, &korobov_a, &merit, &label_y,
                              &label, &sorted_v, &sorted_i, &err, &out_sums, &out_steps,
                              &out_sums64, &out_steps64, &trace_tau, &trace_phi, &diag_x,
                              &diag_it, &diag_st, &stat_counts, &one, &iterstate, &bridge_w,
                              &check_buf};
        for (bap::DevBuf* b : all) f(*b);
    }
};

namespace bap {

bap_status model_prepare(const bap_model* md, DevModel* out);
// Loads every kernel of the library on `device` (the current device) once per process.
bap_status preload_kernels(int device);
bap_status option_alloc(bap_option** out);
bap_status option_load(bap_option* o, const DevModel& hm);
bap_status option_create(const bap_model* md, bap_option** out);
void option_destroy(bap_option* o);
bap_status validate_iz(int d, const bap_iz_params* p);
bap_status validate_cmc(const bap_option* o, const bap_cmc_params* p);
bap_status validate_price(const bap_option* o, int64_t n_paths);
// Enqueue on the option's stream; the matching finish_* reads the results once the stream has
// reached them (after cudaStreamSynchronize or a completed event).
bap_status enqueue_fit_iz(bap_option* o, const bap_iz_params* p);
bap_status finish_fit_iz(bap_option* o);
bap_status enqueue_fit_cmc(bap_option* o, const bap_cmc_params* p);
bap_status finish_fit_cmc(bap_option* o);
bap_status enqueue_price(bap_option* o, int64_t n_paths, uint64_t seed);
bap_status finish_price(bap_option* o, bap_result* res);
// Device memory an option of this model needs for a fit of this size (admission control).
size_t estimate_bytes(const bap_model* md, int method, const void* params, int64_t n_paths);

}  // namespace bap
