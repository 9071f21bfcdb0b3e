// Many independent Taylor-Couette cases on one GPU.
//
// Batch: N cases of any shapes, each with its own resident state and tables,
// stepped together by one CUDA graph whose branches are the cases' kernel
// sequences (launched once per step; the branches run concurrently).
//
// Server: continuous batching.  Requests (case parameters, initial
// perturbation, number of steps) are queued by tc_server_submit from any host
// thread; a worker thread admits them while the estimated device bytes of the
// admitted cases stay within the budget, gives each its own stream, and keeps
// one step in flight per case, relaunching each case as soon as its previous
// step completes, so requests that arrive while others run overlap with them
// on the device.  A finished case is read back (statistics, optional final
// v and eta into caller buffers) and freed, which admits waiting requests.
// Each case's arithmetic is the single-case path, so a result does not depend
// on what else runs.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>

#include "tc_host.h"

using tcx::set_err;

#define CKR(call, ret)                                                            \
    do {                                                                          \
        cudaError_t _e = (call);                                                  \
        if (_e != cudaSuccess) {                                                  \
            set_err(std::string(#call) + ": " + cudaGetErrorString(_e));          \
            return ret;                                                           \
        }                                                                         \
    } while (0)

struct tc_batch {
    std::vector<tc_handle*> cases;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaStream_t root = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t graph = nullptr;
};

static void batch_free(tc_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (auto e : b->joins) cudaEventDestroy(e);
    for (auto s : b->streams) cudaStreamDestroy(s);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->root) cudaStreamDestroy(b->root);
    for (auto h : b->cases) tc_destroy(h);
    delete b;
}

static int batch_graph(tc_batch* b) {
    if (b->graph) return TC_OK;
    const int n = (int)b->cases.size();
    for (int i = 0; i < n; ++i) {
        int rc = tcx::ensure_init(b->cases[i]);
        if (!rc) rc = tcx::prepare_pipeline(b->cases[i]);
        if (rc) return rc;
    }
    CKR(cudaStreamSynchronize(nullptr), TC_ERR_CUDA);
    cudaGraph_t g;
    CKR(cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal), TC_ERR_CUDA);
    CKR(cudaEventRecord(b->fork, b->root), TC_ERR_CUDA);
    for (int i = 0; i < n; ++i) {
        CKR(cudaStreamWaitEvent(b->streams[i], b->fork, 0), TC_ERR_CUDA);
        tcx::launch_step(b->cases[i], b->streams[i]);
        CKR(cudaEventRecord(b->joins[i], b->streams[i]), TC_ERR_CUDA);
        CKR(cudaStreamWaitEvent(b->root, b->joins[i], 0), TC_ERR_CUDA);
    }
    cudaError_t e = cudaStreamEndCapture(b->root, &g);
    if (e != cudaSuccess) { set_err(std::string("batch graph capture: ") + cudaGetErrorString(e)); return TC_ERR_CUDA; }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { set_err(std::string("batch graph instantiate: ") + cudaGetErrorString(e)); return TC_ERR_CUDA; }
    return TC_OK;
}

// ---------------------------------------------------------------------------
namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    long long id;
    tc_params p;
    std::vector<double2> v0, e0;
    int nsteps;
    void* out_v;
    void* out_e;
    size_t need;
    double t_submit;
};

struct Active {
    Request rq;
    tc_handle* h = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int done = 0;
    bool in_flight = false;
    double t_start = 0;
    std::vector<float> lat;
};

float percentile(std::vector<float> v, double q) {
    if (v.empty()) return 0.0f;
    std::sort(v.begin(), v.end());
    size_t i = (size_t)std::min<double>(v.size() - 1, std::max(0.0, q * (v.size() - 1) + 0.5));
    return v[i];
}

}  // namespace

struct tc_server {
    size_t budget = 0, used = 0, peak_used = 0;
    int max_active = 0, device = 0;
    std::deque<Request> queue;
    std::vector<Active*> active;
    std::deque<tc_result> results;
    std::vector<float> all_lat;
    long long next_id = 1, submitted = 0, finished = 0;
    double gp_steps = 0, busy_start = -1, busy_end = 0;
    int peak_active = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    std::string worker_error;
};

namespace {

void finish(tc_server* S, Active* a, int status) {
    tc_result r;
    std::memset(&r, 0, sizeof(r));
    r.id = a->rq.id;
    r.status = status;
    r.steps = a->done;
    if (a->h) {
        if (status == TC_OK) {
            if (tc_torque_stats(a->h, &r.stats) != TC_OK) r.status = TC_ERR_CUDA;
            const size_t nb = tc_field_bytes(a->h, TC_FIELD_V, TC_SPECTRAL);
            if (a->rq.out_v && tc_get_field(a->h, TC_FIELD_V, TC_SPECTRAL, a->rq.out_v, nb) != TC_OK) r.status = TC_ERR_CUDA;
            if (a->rq.out_e && tc_get_field(a->h, TC_FIELD_ETA, TC_SPECTRAL, a->rq.out_e, nb) != TC_OK) r.status = TC_ERR_CUDA;
        }
        tc_destroy(a->h);
    }
    if (a->ev0) cudaEventDestroy(a->ev0);
    if (a->ev1) cudaEventDestroy(a->ev1);
    if (a->s) cudaStreamDestroy(a->s);
    const double t = now_ms();
    r.queue_ms = a->t_start - a->rq.t_submit;
    r.run_ms = t - a->t_start;
    r.step_ms_p50 = percentile(a->lat, 0.50);
    r.step_ms_p99 = percentile(a->lat, 0.99);
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= a->rq.need;
    S->all_lat.insert(S->all_lat.end(), a->lat.begin(), a->lat.end());
    S->gp_steps += (double)a->rq.p.Nr * a->rq.p.Ntheta * a->rq.p.Nz * a->done;
    S->results.push_back(r);
    S->finished++;
    S->busy_end = t;
    delete a;
    S->cv.notify_all();
}

Active* admit(tc_server* S, Request&& rq) {
    Active* a = new Active();
    a->rq = std::move(rq);
    a->t_start = now_ms();
    a->h = tc_create_ex(&a->rq.p);
    int rc = a->h ? TC_OK : TC_ERR_CUDA;
    if (!rc && cudaStreamCreateWithFlags(&a->s, cudaStreamNonBlocking) != cudaSuccess) rc = TC_ERR_CUDA;
    if (!rc && (cudaEventCreate(&a->ev0) != cudaSuccess || cudaEventCreate(&a->ev1) != cudaSuccess)) rc = TC_ERR_CUDA;
    if (!rc) rc = tc_set_stream(a->h, a->s);
    const size_t nb = (size_t)a->rq.p.Nr * a->rq.p.Nz * (a->rq.p.Ntheta / 2) * sizeof(double2);
    if (!rc && !a->rq.v0.empty()) rc = tc_set_field(a->h, TC_FIELD_V, a->rq.v0.data(), nb);
    if (!rc && !a->rq.e0.empty()) rc = tc_set_field(a->h, TC_FIELD_ETA, a->rq.e0.data(), nb);
    if (!rc) rc = tcx::ensure_init(a->h);
    if (!rc) rc = tcx::ensure_graph(a->h);
    a->rq.v0.clear(); a->rq.v0.shrink_to_fit();
    a->rq.e0.clear(); a->rq.e0.shrink_to_fit();
    if (rc) { finish(S, a, rc); return nullptr; }
    return a;
}

void launch_one(Active* a) {
    cudaEventRecord(a->ev0, a->s);
    cudaGraphLaunch(a->h->graph, a->s);
    cudaEventRecord(a->ev1, a->s);
    a->in_flight = true;
}

void worker_main(tc_server* S) {
    if (cudaSetDevice(S->device) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->worker_error = "cudaSetDevice failed in the server worker";
        return;
    }
    for (;;) {
        std::vector<Request> to_admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            while (!S->queue.empty() && (int)(S->active.size() + to_admit.size()) < S->max_active &&
                   S->used + S->queue.front().need <= S->budget) {
                S->used += S->queue.front().need;
                S->peak_used = std::max(S->peak_used, S->used);
                to_admit.push_back(std::move(S->queue.front()));
                S->queue.pop_front();
            }
            if (S->stop && S->queue.empty() && S->active.empty() && to_admit.empty()) break;
            if (S->active.empty() && to_admit.empty()) {
                S->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        for (auto& rq : to_admit) {
            Active* a = admit(S, std::move(rq));
            if (a) {
                if (S->busy_start < 0) S->busy_start = a->t_start;
                S->active.push_back(a);
                launch_one(a);
            }
        }
        S->peak_active = std::max(S->peak_active, (int)S->active.size());
        // poll: relaunch every case whose step has completed
        bool progressed = false;
        for (size_t i = 0; i < S->active.size();) {
            Active* a = S->active[i];
            cudaError_t q = cudaEventQuery(a->ev1);
            if (q == cudaErrorNotReady) { ++i; continue; }
            progressed = true;
            float ms = 0;
            if (q == cudaSuccess) cudaEventElapsedTime(&ms, a->ev0, a->ev1);
            a->in_flight = false;
            a->lat.push_back(ms);
            a->done++;
            a->h->t += a->h->d.dt;
            a->h->step += 1;
            int st = (q == cudaSuccess) ? TC_OK : TC_ERR_CUDA;
            bool stopping;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                stopping = S->stop;
            }
            if (st == TC_OK && (a->done >= a->rq.nsteps || stopping)) st = tcx::check_flags(a->h);
            if (st != TC_OK || a->done >= a->rq.nsteps || stopping) {
                S->active.erase(S->active.begin() + i);
                finish(S, a, st);
                continue;
            }
            launch_one(a);
            ++i;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

size_t tc_estimate_device_bytes(const tc_params* p) {
    if (!p || tcx::validate(p)) return 0;
    return tcx::estimate_device_bytes(*p);
}

tc_batch* tc_batch_create(int ncases, const tc_params* params) {
    if (ncases < 1 || !params) { set_err("tc_batch_create: need ncases >= 1 and parameters"); return nullptr; }
    tc_batch* b = new tc_batch();
    for (int i = 0; i < ncases; ++i) {
        tc_handle* h = tc_create_ex(&params[i]);
        if (!h) {
            std::string msg = "case " + std::to_string(i) + ": " + tc_last_error();
            batch_free(b);
            set_err(msg);
            return nullptr;
        }
        b->cases.push_back(h);
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            batch_free(b);
            set_err("tc_batch_create: stream/event creation failed");
            return nullptr;
        }
        b->streams.push_back(s);
        b->joins.push_back(e);
    }
    if (cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        batch_free(b);
        set_err("tc_batch_create: stream/event creation failed");
        return nullptr;
    }
    return b;
}

tc_handle* tc_batch_case(tc_batch* b, int i) {
    if (!b || i < 0 || i >= (int)b->cases.size()) { set_err("tc_batch_case: index out of range"); return nullptr; }
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }   // the caller may change the case
    return b->cases[i];
}

int tc_batch_step(tc_batch* b, int nsteps) {
    if (!b || nsteps < 0) { set_err("tc_batch_step: invalid arguments"); return TC_ERR_ARG; }
    for (auto h : b->cases)
        if (h->phase != 0) { set_err("tc_batch_step: a case is inside a step"); return TC_ERR_ARG; }
    int rc = batch_graph(b);
    if (rc) return rc;
    for (int n = 0; n < nsteps; ++n) CKR(cudaGraphLaunch(b->graph, b->root), TC_ERR_CUDA);
    CKR(cudaStreamSynchronize(b->root), TC_ERR_CUDA);
    for (auto h : b->cases) {
        h->t += nsteps * h->d.dt;
        h->step += nsteps;
    }
    for (auto h : b->cases) {
        rc = tcx::check_flags(h);
        if (rc) return rc;
    }
    return TC_OK;
}

int tc_batch_set_stream(tc_batch* b, void* stream) {
    if (!b) { set_err("null batch"); return TC_ERR_ARG; }
    // the graph is launched on the root stream; make the caller's stream the root
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    if (b->root) cudaStreamDestroy(b->root);
    b->root = nullptr;
    if (stream) { b->root = (cudaStream_t)stream; return TC_OK; }
    CKR(cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking), TC_ERR_CUDA);
    return TC_OK;
}

size_t tc_batch_device_bytes(const tc_batch* b) {
    size_t s = 0;
    if (b) for (auto h : b->cases) s += tc_device_bytes(h);
    return s;
}

void tc_batch_destroy(tc_batch* b) {
    if (!b) return;
    if (b->root) cudaStreamSynchronize(b->root);
    batch_free(b);
}

tc_server* tc_server_create(size_t budget_bytes, int max_active, int device) {
    if (budget_bytes == 0 || max_active < 1) { set_err("tc_server_create: budget and max_active must be positive"); return nullptr; }
    tc_server* S = new tc_server();
    S->budget = budget_bytes;
    S->max_active = max_active;
    if (device < 0) {
        if (cudaGetDevice(&S->device) != cudaSuccess) { delete S; set_err("cudaGetDevice failed"); return nullptr; }
    } else {
        S->device = device;
    }
    S->worker = std::thread(worker_main, S);
    return S;
}

int tc_server_submit(tc_server* S, const tc_params* p, const void* v0, const void* eta0, int nsteps,
                     void* out_v, void* out_eta, long long* id) {
    if (!S || !p || nsteps < 1) { set_err("tc_server_submit: invalid arguments"); return TC_ERR_ARG; }
    int rc = tcx::validate(p);
    if (rc) return rc;
    Request rq;
    rq.p = *p;
    rq.p.device = S->device;
    rq.nsteps = nsteps;
    rq.out_v = out_v;
    rq.out_e = out_eta;
    rq.need = tcx::estimate_device_bytes(*p);
    if (rq.need > S->budget) { set_err("tc_server_submit: the case alone exceeds the device budget"); return TC_ERR_SIZE; }
    const size_t n = (size_t)p->Nr * p->Nz * (p->Ntheta / 2);
    if (v0) rq.v0.assign((const double2*)v0, (const double2*)v0 + n);
    if (eta0) rq.e0.assign((const double2*)eta0, (const double2*)eta0 + n);
    rq.t_submit = now_ms();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) { set_err("tc_server_submit: server is stopping"); return TC_ERR_ARG; }
    rq.id = S->next_id++;
    if (id) *id = rq.id;
    S->queue.push_back(std::move(rq));
    S->submitted++;
    S->cv.notify_all();
    return TC_OK;
}

int tc_server_poll(tc_server* S, tc_result* out, int max_results, int* count) {
    if (!S || !count || (max_results > 0 && !out)) { set_err("tc_server_poll: invalid arguments"); return TC_ERR_ARG; }
    std::lock_guard<std::mutex> lk(S->mu);
    int n = 0;
    while (n < max_results && !S->results.empty()) {
        out[n++] = S->results.front();
        S->results.pop_front();
    }
    *count = n;
    if (!S->worker_error.empty()) { set_err(S->worker_error); return TC_ERR_CUDA; }
    return TC_OK;
}

int tc_server_drain(tc_server* S, double timeout_s) {
    if (!S) { set_err("null server"); return TC_ERR_ARG; }
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (S->finished < S->submitted) {
        if (!S->worker_error.empty()) { set_err(S->worker_error); return TC_ERR_CUDA; }
        if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout && S->finished < S->submitted) {
            set_err("tc_server_drain: timed out");
            return TC_ERR_TIMEOUT;
        }
    }
    return TC_OK;
}

int tc_server_stats(tc_server* S, tc_server_stats_t* out) {
    if (!S || !out) { set_err("tc_server_stats: invalid arguments"); return TC_ERR_ARG; }
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->finished = S->finished;
    out->queued = (long long)S->queue.size();
    out->active = (long long)S->active.size();
    out->peak_active = S->peak_active;
    out->budget_bytes = S->budget;
    out->used_bytes = S->used;
    out->peak_used_bytes = S->peak_used;
    out->gridpoint_steps = S->gp_steps;
    out->busy_ms = S->busy_start >= 0 ? S->busy_end - S->busy_start : 0.0;
    out->step_ms_p50 = percentile(S->all_lat, 0.50);
    out->step_ms_p99 = percentile(S->all_lat, 0.99);
    out->steps = (long long)S->all_lat.size();
    return TC_OK;
}

void tc_server_destroy(tc_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->submitted -= (long long)S->queue.size();     // queued requests are dropped
        S->queue.clear();
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    delete S;
}

}  // extern "C"
