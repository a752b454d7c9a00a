// Request loop for repeated scans (include/piccs_server.h): per-patient
// device sessions admitted by HBM footprint, continuous batching of a
// patient's queued scans into one batched reconstruction, several batches in
// flight on their own streams, CUDA-graph replay of each launch sequence.
//
// Threads: callers only touch the queues under `mu`; one worker thread owns
// every session and issues all CUDA work.  A batch's completion is signalled
// by a host function enqueued behind its last copy, which wakes the worker.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "../../include/piccs_server.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    long long id = 0;
    int patient = 0;
    const void *h_proj = nullptr;  // FP32, or BF16 for PICCS_STORAGE_BF16 requests
    float *h_out = nullptr;
    piccs_params params{};
    Clock::time_point t_submit, t_issue, t_done;
    int status = PICCS_OK;
    int batch = 0;
    bool done = false;
    double est_ms = 1.0;  // estimated device time of the scan alone
};

struct Session {
    int patient = 0;
    piccs_geometry geo{};
    std::vector<double> angles;
    std::vector<float> prior;
    size_t bytes = 0;  // device bytes held while resident
    piccs_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::deque<Request *> queue;
    std::vector<Request *> running;
    bool finished = false;  // set by the completion host function (under mu)
    long long last_used = 0;
    long long unit = 0;     // issue unit of the running batch (shared by a group's sessions)
    double unit_ms = 0.0;   // estimated device time per scan of that whole unit
};

struct PendingPatient {
    int patient;
    piccs_geometry geo;
    std::vector<double> angles;
    std::vector<float> prior;
};

thread_local std::string g_create_err;

}  // namespace

struct piccs_server {
    piccs_server_config cfg{};
    int device = 0;
    std::string err;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::set<int> registered;                 // under mu
    std::deque<PendingPatient> new_patients;  // under mu
    std::deque<Request *> incoming;           // under mu
    std::map<long long, Request *> requests;  // under mu
    bool stop = false;                        // under mu
    bool wake = false;                        // under mu
    long long next_id = 1;                    // under mu
    piccs_server_stats st{};                  // under mu
    std::map<int, Session> sessions;          // worker only
    long long tick = 0;                       // worker only
    std::thread worker;
};

namespace {

int fail(piccs_server *srv, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (srv) {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->err = buf;
    } else {
        g_create_err = buf;
    }
    return code;
}

struct DoneArg {
    piccs_server *srv;
    Session *ses;
};

// Runs on a CUDA driver thread once a batch's last copy has finished: no
// CUDA calls here, only the wake-up.
void CUDART_CB batch_done(void *p)
{
    DoneArg *a = static_cast<DoneArg *>(p);
    {
        std::lock_guard<std::mutex> lk(a->srv->mu);
        a->ses->finished = true;
        a->srv->wake = true;
    }
    a->srv->cv_work.notify_one();
    delete a;
}

void finish_requests(piccs_server *srv, std::vector<Request *> &reqs, int status_if_unset)
{
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (Request *r : reqs) {
            if (r->status == PICCS_OK && status_if_unset != PICCS_OK) r->status = status_if_unset;
            r->t_done = now;
            r->done = true;
            if (r->status == PICCS_OK) srv->st.completed += 1;
            else srv->st.failed += 1;
        }
    }
    reqs.clear();
    srv->cv_done.notify_all();
}

void evict(piccs_server *srv, Session &s)
{
    if (!s.ctx) return;
    piccs_destroy(s.ctx);
    cudaStreamDestroy(s.stream);
    s.ctx = nullptr;
    s.stream = nullptr;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->st.hbm_in_use -= s.bytes;
    s.bytes = 0;
}

// Makes the session resident with room for `params` (creating it, evicting
// idle sessions if the budget requires).  Returns PICCS_OK, 1 if it has to
// wait for memory to free up, or an error.
int make_resident(piccs_server *srv, Session &s, const piccs_params &params)
{
    size_t need = 0;
    int rc = piccs_query_workspace_batched(&s.geo, &params, srv->cfg.max_batch, &need);
    if (rc != PICCS_OK) return rc;
    if (s.ctx && need <= s.bytes) return PICCS_OK;
    size_t used;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        used = srv->st.hbm_in_use;
    }
    const size_t extra = need - s.bytes;
    while (used + extra > srv->cfg.hbm_budget) {
        Session *lru = nullptr;
        for (auto &kv : srv->sessions) {
            Session &o = kv.second;
            if (&o == &s || !o.ctx || !o.running.empty() || !o.queue.empty()) continue;
            if (!lru || o.last_used < lru->last_used) lru = &o;
        }
        if (!lru) return 1;
        const size_t freed = lru->bytes;
        evict(srv, *lru);
        used -= freed;
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->st.evictions += 1;
    }
    if (!s.ctx) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return PICCS_ECUDA;
        }
        rc = piccs_create_batched(&s.ctx, &s.geo, srv->cfg.max_batch, s.stream);
        if (rc == PICCS_OK) rc = piccs_set_prior_broadcast(s.ctx, s.prior.data(), 1);
        if (rc != PICCS_OK) {
            if (s.ctx) piccs_destroy(s.ctx);
            cudaStreamDestroy(s.stream);
            s.ctx = nullptr;
            s.stream = nullptr;
            return rc;
        }
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->st.sessions_made += 1;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->st.hbm_in_use += extra;
    s.bytes = need;
    return PICCS_OK;
}

// Device time of one scan, from its size: every iteration projects each ray
// through about (nx + ny) / 2 voxels twice (A and A^T, ~1.2e9 pieces per ms)
// and streams the volume's vectors a few times (~20 pieces' worth per voxel).
double estimate_ms(const piccs_geometry &g, const piccs_params &p)
{
    const double N = (double)g.n_views * g.nu * g.nv, M = (double)g.nx * g.ny * g.nz;
    const double its = (double)p.n_outer * (p.n_inner > 0 ? p.n_inner : 0) + 1.0;
    return its * (N * (g.nx + g.ny) + 20.0 * M) / 1.2e9;
}

// A scan whose estimated device time reaches this fills the GPU on its own:
// running a second batch beside it only stretches both.
constexpr double kOverlapMs = 25.0;

// Graphs pay off where launches cost a noticeable part of a scan; for longer
// scans the one-time capture of a new (parameters, batch size) pair would
// only delay the batch.
constexpr double kGraphMs = 200.0;

bool same_params(const piccs_params &a, const piccs_params &b)
{
    return std::memcmp(&a, &b, sizeof a) == 0;
}

// Issues the batches of sessions g[0..n) as one unit: one session's batch,
// or (n > 1) a group -- sessions of different patients whose head requests
// share parameters, run together by piccs_run_staged_group.  Sessions that
// have to wait for memory are left out; false if none could be issued.
// backlog: requests queued over all sessions.
bool issue_unit(piccs_server *srv, Session *const *g, int n, int backlog)
{
    // make every member resident first (their queues are still full, so
    // admitting one cannot evict another)
    std::vector<Session *> ready;
    bool issued = false;
    for (int i = 0; i < n; ++i) {
        Session &s = *g[i];
        Request *head = s.queue.front();
        const int rc = make_resident(srv, s, head->params);
        if (rc == 1) continue;
        if (rc != PICCS_OK) {  // this request cannot run: fail it alone
            s.queue.pop_front();
            head->status = rc;
            std::vector<Request *> one{head};
            finish_requests(srv, one, rc);
            issued = true;
            continue;
        }
        ready.push_back(&s);
    }
    if (ready.empty()) return issued;
    const piccs_params params = ready[0]->queue.front()->params;
    // A long scan gains little from sharing launches (the GPU is full either
    // way) while the first scan of a batch waits for the whole batch: long
    // scans are batched only to work off a deep backlog.
    std::vector<std::vector<Request *>> batches(ready.size());
    bool graph = srv->cfg.use_graphs != 0;
    double unit_ms = 0.0;
    int rc = PICCS_OK;
    const auto now = Clock::now();
    for (size_t m = 0; m < ready.size(); ++m) {
        Session &s = *ready[m];
        Request *head = s.queue.front();
        const int cap = head->est_ms < kGraphMs || backlog > 2 * srv->cfg.max_batch ? srv->cfg.max_batch : 1;
        for (auto it = s.queue.begin(); it != s.queue.end() && (int)batches[m].size() < cap;) {
            if (same_params((*it)->params, params)) {
                batches[m].push_back(*it);
                it = s.queue.erase(it);
            } else {
                ++it;
            }
        }
        graph = graph && head->est_ms < kGraphMs;
        unit_ms += head->est_ms;
        const int nb = (int)batches[m].size();
        for (int i = 0; i < nb; ++i) {
            batches[m][i]->t_issue = now;
            batches[m][i]->batch = nb;
            if (rc == PICCS_OK)
                rc = params.storage == PICCS_STORAGE_BF16
                         ? piccs_stage_bf16(s.ctx, i, batches[m][i]->h_proj, 1)
                         : piccs_stage(s.ctx, i, static_cast<const float *>(batches[m][i]->h_proj), 1);
        }
    }
    const int nm = (int)ready.size();
    piccs_ctx *ctxs[8];
    int nact[8];
    for (int m = 0; m < nm; ++m) {
        ctxs[m] = ready[m]->ctx;
        nact[m] = (int)batches[m].size();
    }
    if (rc == PICCS_OK) rc = piccs_run_staged_group(ctxs, nact, nm, &params, graph);
    for (int m = 0; m < nm && rc == PICCS_OK; ++m)
        for (int i = 0; i < nact[m] && rc == PICCS_OK; ++i)
            rc = piccs_unstage(ready[m]->ctx, i, batches[m][i]->h_out, 1);
    for (int m = 0; m < nm && rc == PICCS_OK; ++m) {
        DoneArg *a = new (std::nothrow) DoneArg{srv, ready[m]};
        if (!a || cudaLaunchHostFunc(ready[m]->stream, batch_done, a) != cudaSuccess) {
            delete a;
            cudaGetLastError();
            rc = PICCS_ECUDA;
        }
    }
    if (rc != PICCS_OK) {  // the sessions' state is unknown: drop them, they are re-created on demand
        for (int m = 0; m < nm; ++m) {
            Session &s = *ready[m];
            if (s.stream) cudaStreamSynchronize(s.stream);
            s.running.clear();
            evict(srv, s);
            finish_requests(srv, batches[m], rc);
        }
        return true;
    }
    const long long unit = ++srv->tick;
    for (int m = 0; m < nm; ++m) {
        Session &s = *ready[m];
        s.running = std::move(batches[m]);
        s.last_used = unit;
        s.unit = unit;
        s.unit_ms = unit_ms;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->st.batches += nm;
    if (graph) srv->st.graph_replays += 1;
    if (nm > 1) srv->st.group_runs += 1;
    return true;
}

void collect(piccs_server *srv, Session &s)
{
    for (int i = 0; i < (int)s.running.size(); ++i) {
        piccs_stats rep;
        int rc = piccs_report_slot(s.ctx, i, &rep);
        s.running[i]->status = rc != PICCS_OK ? rc : rep.status;
    }
    finish_requests(srv, s.running, PICCS_OK);
}

void worker_main(piccs_server *srv)
{
    cudaSetDevice(srv->device);
    bool in_flight = false;
    for (;;) {
        std::deque<Request *> arrived;
        std::deque<PendingPatient> patients;
        std::vector<Session *> finished;
        bool stopping;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            // a stopping server still waits for the completions of its batches
            srv->cv_work.wait(lk, [&] { return srv->wake || (srv->stop && !in_flight); });
            srv->wake = false;
            arrived.swap(srv->incoming);
            patients.swap(srv->new_patients);
            for (auto &kv : srv->sessions)
                if (kv.second.finished) {
                    kv.second.finished = false;
                    finished.push_back(&kv.second);
                }
            stopping = srv->stop;
        }
        for (auto &pp : patients) {
            Session &s = srv->sessions[pp.patient];
            s.patient = pp.patient;
            s.angles = std::move(pp.angles);
            s.geo = pp.geo;
            s.geo.angles_rad = s.angles.data();
            s.prior = std::move(pp.prior);
        }
        for (Request *r : arrived) {
            Session &s = srv->sessions[r->patient];
            r->est_ms = estimate_ms(s.geo, r->params);
            s.queue.push_back(r);
        }
        for (Session *s : finished) collect(srv, *s);

        // issue: highest response ratio (waited + estimated run) / estimated
        // run first -- short scans go ahead of long ones, and a long scan's
        // ratio grows while it waits, so none waits without bound
        // in flight: issue units (a group's sessions share one)
        int running = 0;
        bool big_running = false;
        {
            std::set<long long> units;
            for (auto &kv : srv->sessions)
                if (!kv.second.running.empty() && units.insert(kv.second.unit).second) {
                    running += 1;
                    big_running |= kv.second.unit_ms >= kOverlapMs;
                }
        }
        int backlog = 0;
        for (auto &kv : srv->sessions) backlog += (int)kv.second.queue.size();
        const bool by_ratio = srv->cfg.order == PICCS_ORDER_RESPONSE_RATIO ||
                              (srv->cfg.order == PICCS_ORDER_ADAPTIVE && backlog > 2 * srv->cfg.max_batch);
        bool progress = true;
        while (progress && running < srv->cfg.max_running) {
            progress = false;
            Session *best = nullptr;
            double best_ratio = -1e300;
            const auto now = Clock::now();
            for (auto &kv : srv->sessions) {
                Session &s = kv.second;
                if (!s.running.empty() || s.queue.empty()) continue;
                const Request *h = s.queue.front();
                const double ratio = !by_ratio ? -(double)h->id  // oldest first
                                               : (ms_between(h->t_submit, now) + h->est_ms) / h->est_ms;
                if (ratio > best_ratio) {
                    best_ratio = ratio;
                    best = &s;
                }
            }
            if (!best) break;
            // a short head scan takes other idle sessions whose head requests
            // share its parameters along, in issue order, as one group
            std::vector<Session *> unit{best};
            const Request *bh = best->queue.front();
            if (srv->cfg.max_group > 1 && bh->est_ms < kGraphMs) {
                std::vector<std::pair<double, Session *>> cand;
                for (auto &kv : srv->sessions) {
                    Session &o = kv.second;
                    if (&o == best || !o.running.empty() || o.queue.empty()) continue;
                    const Request *h = o.queue.front();
                    if (h->est_ms >= kGraphMs || !same_params(h->params, bh->params)) continue;
                    cand.push_back({!by_ratio ? -(double)h->id
                                              : (ms_between(h->t_submit, now) + h->est_ms) / h->est_ms,
                                    &o});
                }
                std::stable_sort(cand.begin(), cand.end(),
                                 [](const std::pair<double, Session *> &a, const std::pair<double, Session *> &b) {
                                     return a.first > b.first;
                                 });
                for (auto &c : cand) {
                    if ((int)unit.size() >= srv->cfg.max_group) break;
                    unit.push_back(c.second);
                }
            }
            double unit_ms = 0.0;
            for (Session *u : unit) unit_ms += u->queue.front()->est_ms;
            // batches overlap only while every one of them is small; the order
            // is kept: nothing overtakes a large scan that is next
            if (running > 0 && (big_running || unit_ms >= kOverlapMs)) break;
            if (issue_unit(srv, unit.data(), (int)unit.size(), backlog)) {
                progress = true;
                bool any = false;
                for (Session *u : unit)
                    if (!u->running.empty()) {
                        any = true;
                        big_running |= u->unit_ms >= kOverlapMs;
                    }
                if (any) running += 1;
            } else {
                // wait for memory: try sessions that are already resident
                for (auto &kv : srv->sessions) {
                    Session &s = kv.second;
                    if (&s == best || !s.running.empty() || s.queue.empty() || !s.ctx) continue;
                    if (running > 0 && (big_running || s.queue.front()->est_ms >= kOverlapMs)) continue;
                    Session *one = &s;
                    if (issue_unit(srv, &one, 1, backlog)) {
                        progress = true;
                        if (!s.running.empty()) {
                            running += 1;
                            big_running |= s.unit_ms >= kOverlapMs;
                        }
                        break;
                    }
                }
            }
        }
        bool idle = true;
        for (auto &kv : srv->sessions)
            if (!kv.second.running.empty() || !kv.second.queue.empty()) idle = false;
        in_flight = running > 0;
        if (stopping && idle) {
            std::lock_guard<std::mutex> lk(srv->mu);
            if (srv->incoming.empty() && srv->new_patients.empty()) break;
        }
        if (!idle && running == 0) {
            // queued work that cannot be admitted and nothing running to free memory
            for (auto &kv : srv->sessions) {
                Session &s = kv.second;
                std::vector<Request *> stuck(s.queue.begin(), s.queue.end());
                s.queue.clear();
                finish_requests(srv, stuck, PICCS_ENOMEM);
            }
        }
    }
    for (auto &kv : srv->sessions) evict(srv, kv.second);
}

}  // namespace

extern "C" {

const char *piccs_server_last_error(const piccs_server *srv)
{
    if (!srv) return g_create_err.c_str();
    // the message may be replaced by another thread: hand out a per-thread copy
    thread_local std::string copy;
    std::lock_guard<std::mutex> lk(const_cast<piccs_server *>(srv)->mu);
    copy = srv->err;
    return copy.c_str();
}

int piccs_server_create(piccs_server **out, const piccs_server_config *cfg)
{
    if (!out || !cfg) return fail(nullptr, PICCS_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->max_batch < 1 || cfg->max_batch > 64) return fail(nullptr, PICCS_EINVAL, "max_batch must be in [1, 64]");
    if (cfg->max_running < 1) return fail(nullptr, PICCS_EINVAL, "max_running must be >= 1");
    if (cfg->order < PICCS_ORDER_RESPONSE_RATIO || cfg->order > PICCS_ORDER_ADAPTIVE)
        return fail(nullptr, PICCS_EINVAL, "unknown order %d", cfg->order);
    if (cfg->max_group < 0 || cfg->max_group > 8) return fail(nullptr, PICCS_EINVAL, "max_group must be in [0, 8]");
    piccs_server *srv = new (std::nothrow) piccs_server();
    if (!srv) return fail(nullptr, PICCS_ENOMEM, "host allocation failed");
    srv->cfg = *cfg;
    cudaGetDevice(&srv->device);
    if (srv->cfg.hbm_budget == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            delete srv;
            return fail(nullptr, PICCS_ECUDA, "cudaMemGetInfo failed");
        }
        srv->cfg.hbm_budget = free_b / 10 * 9;
    }
    srv->worker = std::thread(worker_main, srv);
    *out = srv;
    return PICCS_OK;
}

void piccs_server_destroy(piccs_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_one();
    srv->worker.join();
    for (auto &kv : srv->requests) delete kv.second;
    delete srv;
}

int piccs_server_add_patient(piccs_server *srv, int patient, const piccs_geometry *geometry,
                             const float *h_xprior)
{
    if (!srv || !geometry || !h_xprior) return fail(srv, PICCS_EINVAL, "NULL argument");
    int rc = piccs_validate(geometry, nullptr);
    if (rc != PICCS_OK) return fail(srv, rc, "%s", piccs_last_error(nullptr));
    size_t need = 0;
    rc = piccs_query_workspace_batched(geometry, nullptr, srv->cfg.max_batch, &need);
    if (rc != PICCS_OK) return fail(srv, rc, "%s", piccs_last_error(nullptr));
    if (need > srv->cfg.hbm_budget)
        return fail(srv, PICCS_ENOMEM, "session needs %zu bytes, budget %zu", need, srv->cfg.hbm_budget);
    PendingPatient pp;
    pp.patient = patient;
    pp.geo = *geometry;
    pp.angles.assign(geometry->angles_rad, geometry->angles_rad + geometry->n_views);
    const size_t M = (size_t)geometry->nx * geometry->ny * geometry->nz;
    pp.prior.assign(h_xprior, h_xprior + M);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (!srv->registered.insert(patient).second) {
            srv->err = "patient already registered";
            return PICCS_EINVAL;
        }
        srv->new_patients.push_back(std::move(pp));
        srv->wake = true;
    }
    srv->cv_work.notify_one();
    return PICCS_OK;
}

int piccs_server_submit(piccs_server *srv, int patient, const void *h_proj,
                        const piccs_params *params, float *h_out, long long *ticket)
{
    if (!srv || !h_proj || !params || !h_out || !ticket) return fail(srv, PICCS_EINVAL, "NULL argument");
    if (params->x0_mode == PICCS_X0_USER) return fail(srv, PICCS_EINVAL, "requests start from the prior or zero");
    Request *r = new (std::nothrow) Request();
    if (!r) return fail(srv, PICCS_ENOMEM, "host allocation failed");
    r->patient = patient;
    r->h_proj = h_proj;
    r->h_out = h_out;
    r->params = *params;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (!srv->registered.count(patient)) {
            delete r;
            srv->err = "unknown patient";
            return PICCS_EINVAL;
        }
        if (srv->stop) {
            delete r;
            srv->err = "server is stopping";
            return PICCS_EINVAL;
        }
        r->id = srv->next_id++;
        srv->requests[r->id] = r;
        srv->incoming.push_back(r);
        srv->st.submitted += 1;
        srv->wake = true;
        *ticket = r->id;
    }
    srv->cv_work.notify_one();
    return PICCS_OK;
}

int piccs_server_wait(piccs_server *srv, long long ticket, int timeout_ms, piccs_request_stats *st)
{
    if (!srv || !st) return fail(srv, PICCS_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->requests.find(ticket);
    if (it == srv->requests.end()) {
        srv->err = "unknown ticket";
        return PICCS_EINVAL;
    }
    Request *r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) {
        srv->cv_done.wait(lk, ready);
    } else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        return PICCS_ETIMEOUT;
    }
    st->status = r->status;
    st->batch = r->batch;
    st->queued_ms = r->batch ? ms_between(r->t_submit, r->t_issue) : ms_between(r->t_submit, r->t_done);
    st->run_ms = r->batch ? ms_between(r->t_issue, r->t_done) : 0.0;
    st->total_ms = ms_between(r->t_submit, r->t_done);
    srv->requests.erase(it);
    delete r;
    return PICCS_OK;
}

int piccs_server_get_stats(piccs_server *srv, piccs_server_stats *out)
{
    if (!srv || !out) return fail(srv, PICCS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->st;
    return PICCS_OK;
}

}  // extern "C"
