// Many independent Taylor-Couette cases on one GPU.
//
// Batch: N cases of any shapes, each with its own resident state and tables,
// stepped together by one CUDA graph per step.  Cases of the same form and
// Fourier grid (any Nr, radius ratio, Re) form a shape class; each
// plane-phase kernel runs once per class over the radial planes of all of its
// cases (the classes as concurrent branches), and the line kernel and the
// mean flow once per precision form over all of its cases, each block
// reading its case's descriptor.
//
// Server: continuous batching.  Requests (case parameters, initial
// perturbation, number of steps) are queued by tc_server_submit from any host
// thread; a worker thread admits them while the estimated device bytes of the
// admitted cases stay within the budget.  Per-case mode (the default): each
// case has its own stream and one step in flight, relaunched as soon as its
// previous step completes.  Grouped mode: every admitted case advances by one
// step in one graph launch of the batch's grouped kernels, and between steps
// finished cases leave and new ones join.  Either way requests
// that arrive while others run overlap with them on the device.  A finished case is read back (statistics, optional final
// v and eta into caller buffers) and freed, which admits waiting requests.
// Each case's arithmetic is the single-case path, so a result does not depend
// on what else runs.
#include <algorithm>
#include <array>
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

// Cases of one shape class (the same form, Ntheta and Nz; any Nr, radius
// ratio, Re, box): their plane kernels, line kernel and mean flow run as one
// launch each, over the radial planes / pairs / profiles of all of them.
struct BatchClass {
    std::vector<int> cases;
    TcDev d0;                       // representative descriptor (shapes, z tile, plans)
    TcDev* ds = nullptr;            // device: one descriptor per case
    int2* ymap = nullptr;           // device: (case, radial plane) per plane-kernel grid row
    int nplanes = 0, maxNr = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t join = nullptr;
};

// Cases of one precision form: their line kernel is one launch over the
// pairs of all of them (cases ordered by decreasing Nr, so that the longest
// radial lines start first), their mean flows one launch with a block each.
struct BatchForm {
    int prec = 0, ncases = 0, nblocks = 0, maxNr = 0;
    TcDev* ds = nullptr;
    int2* bmap = nullptr;           // (case, block within the case) per line-kernel block
    cudaStream_t sl = nullptr, sm = nullptr;
    cudaEvent_t jl = nullptr, jm = nullptr;
};

// A set of cases stepped together: their shape classes and precision forms,
// and the captured graph of one step of all of them (launched on root).
// Used by the batch, and by the server in its grouped mode.
struct Group {
    std::vector<tc_handle*> cases;
    std::vector<BatchClass> classes;
    std::vector<BatchForm> forms;
    cudaStream_t root = nullptr;
    bool own_root = true;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t graph = nullptr;
};

struct tc_batch : Group {};

static void batch_release_classes(Group* b) {
    for (auto& c : b->classes) {
        if (c.ds) cudaFree(c.ds);
        if (c.ymap) cudaFree(c.ymap);
        if (c.join) cudaEventDestroy(c.join);
        if (c.stream) cudaStreamDestroy(c.stream);
    }
    b->classes.clear();
    for (auto& f : b->forms) {
        if (f.ds) cudaFree(f.ds);
        if (f.bmap) cudaFree(f.bmap);
        for (cudaEvent_t e : {f.jl, f.jm}) if (e) cudaEventDestroy(e);
        for (cudaStream_t t : {f.sl, f.sm}) if (t) cudaStreamDestroy(t);
    }
    b->forms.clear();
}

static void batch_free(tc_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    batch_release_classes(b);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->root && b->own_root) cudaStreamDestroy(b->root);
    for (auto h : b->cases) tc_destroy(h);
    delete b;
}

// Group the cases into shape classes and upload each class's descriptors
// and plane map.  A class runs with the z tile its first case was tuned to
// (launch shapes do not change the arithmetic).
static int batch_classes(Group* b) {
    batch_release_classes(b);
    std::vector<std::array<int, 3>> keys;
    for (int i = 0; i < (int)b->cases.size(); ++i) {
        const TcDev& d = b->cases[i]->d;
        const std::array<int, 3> key = {d.prec, d.Nh, d.Nz};
        size_t c = std::find(keys.begin(), keys.end(), key) - keys.begin();
        if (c == keys.size()) {
            keys.push_back(key);
            b->classes.emplace_back();
            b->classes.back().d0 = d;
        }
        b->classes[c].cases.push_back(i);
    }
    for (auto& c : b->classes) {
        std::vector<TcDev> ds;
        std::vector<int2> ym;
        for (int i = 0; i < (int)c.cases.size(); ++i) {
            TcDev d = b->cases[c.cases[i]]->d;
            d.ztile = c.d0.ztile;
            ds.push_back(d);
            for (int r = 0; r < d.Nr; ++r) ym.push_back(make_int2(i, r));
            c.maxNr = std::max(c.maxNr, d.Nr);
        }
        c.nplanes = (int)ym.size();
        CKR(cudaMalloc(&c.ds, ds.size() * sizeof(TcDev)), TC_ERR_CUDA);
        CKR(cudaMalloc(&c.ymap, ym.size() * sizeof(int2)), TC_ERR_CUDA);
        CKR(cudaMemcpy(c.ds, ds.data(), ds.size() * sizeof(TcDev), cudaMemcpyHostToDevice), TC_ERR_CUDA);
        CKR(cudaMemcpy(c.ymap, ym.data(), ym.size() * sizeof(int2), cudaMemcpyHostToDevice), TC_ERR_CUDA);
        CKR(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), TC_ERR_CUDA);
        CKR(cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming), TC_ERR_CUDA);
    }
    const int bs = tc_line_batch_block();
    for (int prec : {TC_PREC_FP64, TC_PREC_MIXED, TC_PREC_DF64}) {
        std::vector<int> idx;
        for (int i = 0; i < (int)b->cases.size(); ++i)
            if (b->cases[i]->d.prec == prec) idx.push_back(i);
        if (idx.empty()) continue;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return b->cases[a]->d.Nr > b->cases[c]->d.Nr; });
        b->forms.emplace_back();
        BatchForm& f = b->forms.back();
        f.prec = prec;
        f.ncases = (int)idx.size();
        std::vector<TcDev> ds;
        std::vector<int2> bm;
        for (int i = 0; i < f.ncases; ++i) {
            const TcDev& d = b->cases[idx[i]]->d;
            ds.push_back(d);
            f.maxNr = std::max(f.maxNr, d.Nr);
            for (int q = 0; q < (d.npairs + bs - 1) / bs; ++q) bm.push_back(make_int2(i, q));
        }
        f.nblocks = (int)bm.size();
        CKR(cudaMalloc(&f.ds, ds.size() * sizeof(TcDev)), TC_ERR_CUDA);
        CKR(cudaMalloc(&f.bmap, bm.size() * sizeof(int2)), TC_ERR_CUDA);
        CKR(cudaMemcpy(f.ds, ds.data(), ds.size() * sizeof(TcDev), cudaMemcpyHostToDevice), TC_ERR_CUDA);
        CKR(cudaMemcpy(f.bmap, bm.data(), bm.size() * sizeof(int2), cudaMemcpyHostToDevice), TC_ERR_CUDA);
        CKR(cudaStreamCreateWithFlags(&f.sl, cudaStreamNonBlocking), TC_ERR_CUDA);
        CKR(cudaStreamCreateWithFlags(&f.sm, cudaStreamNonBlocking), TC_ERR_CUDA);
        CKR(cudaEventCreateWithFlags(&f.jl, cudaEventDisableTiming), TC_ERR_CUDA);
        CKR(cudaEventCreateWithFlags(&f.jm, cudaEventDisableTiming), TC_ERR_CUDA);
    }
    return TC_OK;
}

// One step of every case, per substep: the plane phase of each shape class
// (z inverse, theta rows, z forward, one launch each over all of the
// class's cases; the classes as concurrent branches), then the line phase of
// each precision form (one launch over all of its cases) beside its mean
// flows (one launch).
static int batch_graph(Group* b) {
    if (b->graph) return TC_OK;
    for (auto h : b->cases) {
        int rc = tcx::ensure_init(h);
        if (rc) return rc;
    }
    CKR(cudaDeviceSynchronize(), TC_ERR_CUDA);
    int rc = batch_classes(b);
    if (rc) return rc;
    cudaGraph_t g;
    CKR(cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal), TC_ERR_CUDA);
    CKR(cudaEventRecord(b->fork, b->root), TC_ERR_CUDA);
    for (int k = 0; k < 3; ++k) {
        if (k > 0) CKR(cudaEventRecord(b->fork, b->root), TC_ERR_CUDA);
        for (auto& c : b->classes) {
            CKR(cudaStreamWaitEvent(c.stream, b->fork, 0), TC_ERR_CUDA);
            for (int w = 0; w < 3; ++w) tc_launch_plane_kernel_batch(c.d0, c.ds, c.ymap, c.nplanes, w, c.stream);
            CKR(cudaEventRecord(c.join, c.stream), TC_ERR_CUDA);
            CKR(cudaStreamWaitEvent(b->root, c.join, 0), TC_ERR_CUDA);
        }
        CKR(cudaEventRecord(b->fork, b->root), TC_ERR_CUDA);
        for (auto& f : b->forms) {
            CKR(cudaStreamWaitEvent(f.sl, b->fork, 0), TC_ERR_CUDA);
            CKR(cudaStreamWaitEvent(f.sm, b->fork, 0), TC_ERR_CUDA);
            tc_launch_line_batch(f.prec, f.ds, f.bmap, f.nblocks, k, f.sl);
            tc_launch_mean_batch(f.prec, f.ds, f.ncases, f.maxNr, k, f.sm);
            CKR(cudaEventRecord(f.jl, f.sl), TC_ERR_CUDA);
            CKR(cudaEventRecord(f.jm, f.sm), TC_ERR_CUDA);
            CKR(cudaStreamWaitEvent(b->root, f.jl, 0), TC_ERR_CUDA);
            CKR(cudaStreamWaitEvent(b->root, f.jm, 0), TC_ERR_CUDA);
        }
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
    int mode = TC_SERVE_PER_CASE;
    cudaStream_t gstream = nullptr;   // grouped mode: the stream of every admitted case
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
    const bool grouped = S->mode == TC_SERVE_GROUPED;
    if (grouped) {
        if (!rc) rc = tc_set_stream(a->h, S->gstream);
    } else {
        if (!rc && cudaStreamCreateWithFlags(&a->s, cudaStreamNonBlocking) != cudaSuccess) rc = TC_ERR_CUDA;
        if (!rc && (cudaEventCreate(&a->ev0) != cudaSuccess || cudaEventCreate(&a->ev1) != cudaSuccess)) rc = TC_ERR_CUDA;
        if (!rc) rc = tc_set_stream(a->h, a->s);
    }
    const size_t nb = (size_t)a->rq.p.Nr * a->rq.p.Nz * (a->rq.p.Ntheta / 2) * sizeof(double2);
    if (!rc && !a->rq.v0.empty()) rc = tc_set_field(a->h, TC_FIELD_V, a->rq.v0.data(), nb);
    if (!rc && !a->rq.e0.empty()) rc = tc_set_field(a->h, TC_FIELD_ETA, a->rq.e0.data(), nb);
    if (!rc) rc = tcx::ensure_init(a->h);
    if (!rc && !grouped) rc = tcx::ensure_graph(a->h);
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

// Grouped mode: every admitted case steps in one graph launch per step (the
// batch's grouped kernels over the current set of cases, captured again
// whenever the set changes); between steps, finished cases leave and queued
// requests are admitted.
void worker_grouped(tc_server* S) {
    Group G;
    G.own_root = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&G.root, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&G.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->worker_error = "stream/event creation failed in the server worker";
        return;
    }
    S->gstream = G.root;
    bool dirty = true;
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
                dirty = true;
            }
        }
        S->peak_active = std::max(S->peak_active, (int)S->active.size());
        if (S->active.empty()) continue;
        int rc = TC_OK;
        if (dirty) {
            if (G.graph) { cudaGraphExecDestroy(G.graph); G.graph = nullptr; }
            batch_release_classes(&G);
            G.cases.clear();
            for (Active* a : S->active) G.cases.push_back(a->h);
            rc = batch_graph(&G);
            dirty = false;
        }
        float ms = 0;
        if (!rc) {
            cudaEventRecord(e0, G.root);
            cudaGraphLaunch(G.graph, G.root);
            cudaEventRecord(e1, G.root);
            rc = cudaEventSynchronize(e1) == cudaSuccess ? TC_OK : TC_ERR_CUDA;
            if (!rc) cudaEventElapsedTime(&ms, e0, e1);
        }
        bool stopping;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            stopping = S->stop;
        }
        for (size_t i = 0; i < S->active.size();) {
            Active* a = S->active[i];
            int st = rc;
            if (!rc) {
                a->lat.push_back(ms);
                a->done++;
                a->h->t += a->h->d.dt;
                a->h->step += 1;
                if (a->done >= a->rq.nsteps || stopping) st = tcx::check_flags(a->h);
            }
            if (st != TC_OK || a->done >= a->rq.nsteps || stopping) {
                S->active.erase(S->active.begin() + i);
                finish(S, a, st);
                dirty = true;
                continue;
            }
            ++i;
        }
    }
    if (G.graph) cudaGraphExecDestroy(G.graph);
    G.graph = nullptr;
    batch_release_classes(&G);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(G.fork);
    cudaStreamDestroy(G.root);
}

void worker_main(tc_server* S) {
    if (cudaSetDevice(S->device) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->worker_error = "cudaSetDevice failed in the server worker";
        return;
    }
    if (S->mode == TC_SERVE_GROUPED) {
        worker_grouped(S);
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
    if (b->root && b->own_root) cudaStreamDestroy(b->root);
    b->root = nullptr;
    if (stream) { b->root = (cudaStream_t)stream; b->own_root = false; return TC_OK; }
    CKR(cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking), TC_ERR_CUDA);
    b->own_root = true;
    return TC_OK;
}

int tc_batch_launches_per_step(const tc_batch* b) {
    if (!b) { set_err("null batch"); return TC_ERR_ARG; }
    std::vector<std::array<int, 3>> keys;
    for (auto h : b->cases) {
        const std::array<int, 3> key = {h->d.prec, h->d.Nh, h->d.Nz};
        if (std::find(keys.begin(), keys.end(), key) == keys.end()) keys.push_back(key);
    }
    std::vector<int> precs;
    for (auto h : b->cases)
        if (std::find(precs.begin(), precs.end(), h->d.prec) == precs.end()) precs.push_back(h->d.prec);
    return 3 * (3 * (int)keys.size() + 2 * (int)precs.size());
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
    return tc_server_create_ex(budget_bytes, max_active, device, TC_SERVE_PER_CASE);
}

tc_server* tc_server_create_ex(size_t budget_bytes, int max_active, int device, int mode) {
    if (budget_bytes == 0 || max_active < 1) { set_err("tc_server_create: budget and max_active must be positive"); return nullptr; }
    if (mode != TC_SERVE_GROUPED && mode != TC_SERVE_PER_CASE) { set_err("tc_server_create: unknown mode"); return nullptr; }
    tc_server* S = new tc_server();
    S->budget = budget_bytes;
    S->max_active = max_active;
    S->mode = mode;
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
