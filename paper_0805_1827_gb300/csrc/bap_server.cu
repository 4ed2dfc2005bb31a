// bap_server.cu -- the serving loop behind bap_server_create / bap_submit / bap_poll.
//
// Continuous batching of pricing requests: a server thread admits queued requests while the
// number in flight and their estimated device memory stay within the limits, starts each one on
// its own CUDA stream (the fit -- a CUDA graph for I&Z -- then the pricing, then an event), and
// finishes whichever requests' events have completed, freeing their slots and memory for the
// queue.  Kernels of different requests therefore overlap on the device, and requests that
// arrive while others run join at the next admission.  Each request's computation depends only
// on its own inputs (fixed work split and fixed-order reductions), so its result is bitwise the
// same alone and in any mix.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "bap_host.cuh"

using namespace bap;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

enum ReqState { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2 };

struct Request {
    uint64_t ticket = 0;
    DevModel hm{};                 // validated and prepared at submit
    int method = 0;
    bap_iz_params iz{};
    bap_cmc_params cmc{};
    int64_t n_paths = 0;
    uint64_t seed = 0;
    size_t mem = 0;
    bap_option* opt = nullptr;
    cudaEvent_t done_ev = nullptr;
    int state = Q_QUEUED;
    bool cancel = false;           // bap_cancel on a running request
    bap_status status = BAP_OK;
    std::string err;
    bap_result res{};
    Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct bap_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::vector<Request*> running;                 // touched by the server thread only
    std::vector<bap_option*> free_slots;           // idle options kept for reuse (server thread)
    std::unordered_map<uint64_t, Request*> table;  // all requests not yet collected
    size_t budget = 0, used = 0;
    int max_inflight = 0;
    int device = 0;
    int launch_mode = LAUNCH_COOP;
    bool stop = false;
    uint64_t next_ticket = 1;
    cudaStream_t cancel_stream = nullptr;          // writes device abort flags (server thread)
    bap_server_stats stats{};
    std::thread th;
};

namespace {

// Starts a request on its own stream; false if it failed before anything was enqueued.
// Starts a request on an idle option slot (a new one if none is idle); false if it failed
// before anything was enqueued.
bool start_request(bap_server* s, Request* r) {
    clear_error();
    bap_status st = BAP_OK;
    if (!s->free_slots.empty()) {
        r->opt = s->free_slots.back();
        s->free_slots.pop_back();
    } else {
        st = option_alloc(&r->opt);
    }
    const auto t0 = Clock::now();
    if (st == BAP_OK) st = option_load(r->opt, r->hm);
    const auto t1 = Clock::now();
    if (st == BAP_OK) {
        r->opt->launch_mode = s->launch_mode;
        // cooperative launches on at most an eighth of the device each (measured best on the
        // mixed stream once idle blocks leave between passes: a quarter 79.2, a half 65.2,
        // an eighth 81.2 options/s)
        r->opt->grid_share = std::min(s->max_inflight, 8);
    }
    if (st == BAP_OK)
        st = r->method == BAP_METHOD_IZ ? enqueue_fit_iz(r->opt, &r->iz) : enqueue_fit_cmc(r->opt, &r->cmc);
    const auto t2 = Clock::now();
    if (st == BAP_OK) st = enqueue_price(r->opt, r->n_paths, r->seed);
    const auto t3 = Clock::now();
    s->stats.load_ms += ms_between(t0, t1);
    s->stats.fit_enqueue_ms += ms_between(t1, t2);
    s->stats.price_enqueue_ms += ms_between(t2, t3);
    if (st == BAP_OK && cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming) != cudaSuccess)
        st = fail(BAP_ECUDA, "event create");
    if (st == BAP_OK && cudaEventRecord(r->done_ev, r->opt->stream) != cudaSuccess)
        st = fail(BAP_ECUDA, "event record");
    if (st != BAP_OK) {
        r->status = st;
        r->err = error_text();
        return false;
    }
    return true;
}

void finish_request(Request* r) {
    clear_error();
    bap_status st = r->method == BAP_METHOD_IZ ? finish_fit_iz(r->opt) : finish_fit_cmc(r->opt);
    bap_status sp = finish_price(r->opt, &r->res);
    if (sp != BAP_OK) st = sp;
    r->status = st;
    if (st != BAP_OK && st != BAP_ENOCONV) r->err = error_text();
}

// Returns the request's option to the idle slots (destroys it after a device error).
void release(bap_server* s, Request* r) {
    if (r->done_ev) cudaEventDestroy(r->done_ev);
    r->done_ev = nullptr;
    if (r->opt) {
        if (r->status == BAP_ECUDA) option_destroy(r->opt);
        else s->free_slots.push_back(r->opt);
    }
    r->opt = nullptr;
}

void server_loop(bap_server* s) {
    cudaSetDevice(s->device);
    if (cudaStreamCreateWithFlags(&s->cancel_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        s->cancel_stream = nullptr;
    }
    for (;;) {
        std::vector<Request*> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->queue.empty() && s->running.empty()) break;
            while (!s->queue.empty() && (int)s->running.size() + (int)admit.size() < s->max_inflight) {
                Request* r = s->queue.front();
                const bool fits = s->used + r->mem <= s->budget;
                if (!fits && (!s->running.empty() || !admit.empty())) break;   // wait for memory
                s->queue.pop_front();
                s->used += r->mem;
                r->state = Q_RUNNING;
                r->t_admit = Clock::now();
                admit.push_back(r);
            }
            s->stats.peak_bytes = std::max<int64_t>(s->stats.peak_bytes, (int64_t)s->used);
        }
        for (Request* r : admit) {
            const auto t0 = Clock::now();
            const bool ok = start_request(s, r);
            s->stats.start_ms += ms_between(t0, Clock::now());
            if (ok) {
                s->running.push_back(r);
            } else {
                release(s, r);
                std::lock_guard<std::mutex> lk(s->mu);
                s->used -= r->mem;
                r->state = Q_DONE;
                r->t_done = Clock::now();
                s->stats.failed += 1;
                s->cv_done.notify_all();
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stats.peak_inflight = std::max<int64_t>(s->stats.peak_inflight, (int64_t)s->running.size());
        }
        bool progressed = !admit.empty();
        for (size_t i = 0; i < s->running.size();) {
            Request* r = s->running[i];
            const cudaError_t q = cudaEventQuery(r->done_ev);
            if (q == cudaErrorNotReady) {
                bool cancel;
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    cancel = r->cancel;
                }
                // a cancelled request: keep its abort flag set (the fit's set-up clears it once)
                if (cancel && s->cancel_stream)
                    cudaMemsetAsync(r->opt->stat_counts.as<int>() + 3, 0x01, sizeof(int), s->cancel_stream);
                ++i;
                continue;
            }
            const auto t0 = Clock::now();
            bool cancelled;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                cancelled = r->cancel;
            }
            if (cancelled) {
                if (q != cudaSuccess) cudaGetLastError();
                // no abort-flag write may land after this slot goes to the next request
                if (s->cancel_stream) cudaStreamSynchronize(s->cancel_stream);
                r->status = BAP_ECANCELED;
                r->err = "cancelled";
            } else if (q == cudaSuccess) {
                finish_request(r);
            } else {
                r->status = BAP_ECUDA;
                r->err = cudaGetErrorString(q);
            }
            release(s, r);
            s->stats.finish_ms += ms_between(t0, Clock::now());
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->used -= r->mem;
                r->state = Q_DONE;
                r->t_done = Clock::now();
                if (r->status == BAP_OK || r->status == BAP_ENOCONV) s->stats.completed += 1;
                else s->stats.failed += 1;
                if (r->status == BAP_ECANCELED) s->stats.cancelled += 1;
                s->cv_done.notify_all();
            }
            s->running[i] = s->running.back();
            s->running.pop_back();
            progressed = true;
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->queue.empty() || (int)s->running.size() >= s->max_inflight)
                s->cv_work.wait_for(lk, std::chrono::microseconds(s->running.empty() ? 2000 : 50));
        }
    }
    for (bap_option* o : s->free_slots) option_destroy(o);
    s->free_slots.clear();
    if (s->cancel_stream) {
        cudaStreamSynchronize(s->cancel_stream);
        cudaStreamDestroy(s->cancel_stream);
    }
}

}  // namespace

extern "C" {

bap_status bap_server_create(size_t device_mem_budget, int max_inflight, bap_server** out) {
    clear_error();
    if (!out) return fail(BAP_EINVAL, "null argument");
    *out = nullptr;
    if (device_mem_budget < (1u << 20)) return fail(BAP_EINVAL, "device_mem_budget below 1 MiB");
    if (max_inflight < 1 || max_inflight > 1024) return fail(BAP_EINVAL, "max_inflight outside 1..1024");
    int dev = 0, n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0 || cudaGetDevice(&dev) != cudaSuccess)
        return fail(BAP_ECUDA, "no CUDA device");
    TRY(preload_kernels(dev));
    bap_server* s = new (std::nothrow) bap_server();
    if (!s) return fail(BAP_ENOMEM, "host allocation");
    s->budget = device_mem_budget;
    s->max_inflight = max_inflight;
    s->device = dev;
    try {
        s->th = std::thread(server_loop, s);
    } catch (...) {
        delete s;
        return fail(BAP_ENOMEM, "cannot start the server thread");
    }
    *out = s;
    return BAP_OK;
}

bap_status bap_server_set_launch_mode(bap_server* s, int mode) {
    if (!s) return fail(BAP_EINVAL, "null server");
    if (mode != LAUNCH_PLAIN && mode != LAUNCH_GRAPH && mode != LAUNCH_COOP)
        return fail(BAP_EINVAL, "bad launch mode");
    std::lock_guard<std::mutex> lk(s->mu);
    s->launch_mode = mode;
    return BAP_OK;
}

bap_status bap_submit(bap_server* s, const bap_model* md, int method, const void* params,
                      int64_t n_paths, uint64_t seed, uint64_t* ticket) {
    clear_error();
    if (!s || !md || !params || !ticket) return fail(BAP_EINVAL, "null argument");
    if (method != BAP_METHOD_IZ && method != BAP_METHOD_CMC) return fail(BAP_EINVAL, "bad method");
    if (md->d < 1 || md->d > BAP_MAX_D || md->n_dates < 1 || md->n_dates > BAP_MAX_DATES ||
        !md->S0 || !md->sigma || !md->delta || !md->rho)
        return fail(BAP_EINVAL, "bad model");
    if (n_paths < 2 || n_paths > (1LL << 40)) return fail(BAP_EINVAL, "n_paths outside 2..2^40");
    Request* r = new (std::nothrow) Request();
    if (!r) return fail(BAP_ENOMEM, "host allocation");
    const bap_status sm = model_prepare(md, &r->hm);
    if (sm != BAP_OK) {
        delete r;
        return sm;
    }
    r->method = method;
    bap_status st = BAP_OK;
    if (method == BAP_METHOD_IZ) {
        r->iz = *static_cast<const bap_iz_params*>(params);
        st = validate_iz(r->hm.d, &r->iz);
    } else {
        r->cmc = *static_cast<const bap_cmc_params*>(params);
        st = validate_cmc(nullptr, &r->cmc);
    }
    if (st != BAP_OK) {
        delete r;
        return st;
    }
    r->n_paths = n_paths;
    r->seed = seed;
    r->mem = estimate_bytes(md, method, params, n_paths);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete r;
        return fail(BAP_ESTATE, "server is shutting down");
    }
    if (r->mem > s->budget) {
        const size_t need = r->mem;
        delete r;
        return fail(BAP_EBUSY, "request needs about %zu bytes of device memory; the budget is %zu",
                    need, s->budget);
    }
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->queue.push_back(r);
    s->table[r->ticket] = r;
    s->stats.submitted += 1;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return BAP_OK;
}

static bap_status collect(bap_server* s, std::unordered_map<uint64_t, Request*>::iterator it,
                          bap_result* out) {
    Request* r = it->second;
    const bap_status st = r->status;
    if (out) {
        *out = r->res;
        out->queue_ms = ms_between(r->t_submit, r->t_admit);
        out->latency_ms = ms_between(r->t_submit, r->t_done);
    }
    if (st != BAP_OK && st != BAP_ENOCONV) fail(st, "%s", r->err.c_str());
    s->table.erase(it);
    delete r;
    return st;
}

bap_status bap_poll(bap_server* s, uint64_t ticket, bap_result* out) {
    clear_error();
    if (!s) return fail(BAP_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return fail(BAP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second->state != Q_DONE) return BAP_ENOTREADY;
    return collect(s, it, out);
}

bap_status bap_cancel(bap_server* s, uint64_t ticket) {
    clear_error();
    if (!s) return fail(BAP_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return fail(BAP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Request* r = it->second;
    if (r->state == Q_DONE) return fail(BAP_ESTATE, "request %llu already finished", (unsigned long long)ticket);
    if (r->state == Q_QUEUED) {
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
            if (*q == r) { s->queue.erase(q); break; }
        r->state = Q_DONE;
        r->status = BAP_ECANCELED;
        r->err = "cancelled";
        r->t_admit = r->t_done = Clock::now();
        s->stats.failed += 1;
        s->stats.cancelled += 1;
        s->cv_done.notify_all();
    } else {
        r->cancel = true;
    }
    return BAP_OK;
}

bap_status bap_wait(bap_server* s, uint64_t ticket, double timeout_s, bap_result* out) {
    clear_error();
    if (!s) return fail(BAP_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return fail(BAP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Request* r = it->second;
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (r->state != Q_DONE) {
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && r->state != Q_DONE)
            return fail(BAP_ETIMEOUT, "request %llu not done after %.3f s", (unsigned long long)ticket, timeout_s);
    }
    return collect(s, s->table.find(ticket), out);
}

bap_status bap_server_get_stats(bap_server* s, bap_server_stats* out) {
    if (!s || !out) return fail(BAP_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->queued = (int64_t)s->queue.size();
    out->bytes_in_use = (int64_t)s->used;
    return BAP_OK;
}

void bap_server_destroy(bap_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    for (auto& kv : s->table) delete kv.second;
    delete s;
}

}  // extern "C"
