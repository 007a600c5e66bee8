// server.cu -- a continuous-batching request server over one context.
//
// Requests (a mesh and a chart-solve order/tolerance) are queued in arrival
// order.  A fixed number of worker slots, each a host thread with its own
// CUDA stream, take requests from the head of the queue as soon as a slot is
// free and the request's estimated device footprint fits in the HBM budget
// next to the requests already running.  Each admitted request is uploaded
// (its resident state stays on the device while it runs), solved with
// lsm_solve_charts on its slot's stream, copied back and freed; requests on
// different slots overlap on the GPU.  Results stay with the server until
// the caller releases them.
#include <chrono>
#include <condition_variable>
#include <algorithm>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include "lsm_internal.cuh"

struct lsm_server;

namespace lsm {
namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    int64_t ticket = 0;
    std::vector<double> verts;
    std::vector<int32_t> tris;
    std::vector<double> sigma;
    lsm_quad rule{4, 0};
    int order = 8, max_iter = 20, precision = LSM_MIXED;
    double tol = 1e-10;
    int64_t bytes = 0;
    // result
    int status = LSM_E_NOT_CONVERGED;
    bool done = false;
    double t_submit = 0, t_start = 0, t_done = 0;
    lsm_solve_stats stats{};
    std::vector<double> x, h;
    std::vector<int32_t> node_status;
    std::string err;
};

// Device bytes a request holds while it runs: the mesh's resident state and
// the chart solve's node state and scratch.
int64_t footprint(int64_t nv, int64_t nt, int nq, int n_gl)
{
    const int64_t ns = nt * nq;
    const int64_t nodes = nt * (int64_t)n_gl * n_gl;
    return ns * 144 + nt * 64 + nv * 48 + nodes * 260 + (int64_t)(64 << 20) / 16;
}

}  // namespace
}  // namespace lsm

struct lsm_server {
    lsm_ctx* ctx = nullptr;
    int64_t budget = 0;
    int64_t in_use = 0;
    int64_t next_ticket = 1;
    bool stopping = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<lsm::Job>> queue;
    std::map<int64_t, std::shared_ptr<lsm::Job>> jobs;
    std::vector<std::thread> workers;
    lsm::Clock::time_point t0;
    int64_t peak_in_use = 0;
    int max_running = 0, running = 0;
};

namespace lsm {
namespace {

double ms_since(const lsm_server* s) {
    return std::chrono::duration<double, std::milli>(Clock::now() - s->t0).count();
}

void run_job(lsm_server* sv, cudaStream_t st, Job& j)
{
    lsm_mesh* mesh = nullptr;
    int rc = lsm_mesh_upload(sv->ctx, j.verts.data(), (int64_t)(j.verts.size() / 3), j.tris.data(),
                             (int64_t)(j.tris.size() / 3), j.sigma.empty() ? nullptr : j.sigma.data(), &j.rule, st,
                             &mesh);
    if (rc == LSM_OK) {
        const int n_gl = j.order / 2 + 2;
        const size_t n = j.tris.size() / 3 * (size_t)n_gl * n_gl;
        j.x.resize(3 * n);
        j.h.resize(n);
        j.node_status.resize(n);
        rc = lsm_solve_charts(mesh, j.order, j.tol, j.max_iter, j.precision, j.x.data(), j.h.data(),
                              j.node_status.data(), &j.stats, st);
    }
    // the message this worker thread's own failing call recorded
    if (rc != LSM_OK) j.err = lsm_last_error(sv->ctx);
    if (mesh) lsm_mesh_free(mesh);
    j.status = rc;
}

void worker(lsm_server* sv)
{
    cudaSetDevice(sv->ctx->c.device);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
    // this slot's own device error word: a wait that runs out in one request
    // is charged to that request, not to whichever slot checks the word first
    // (the messages are per thread already)
    int* wflag = nullptr;
    if (cudaMalloc(&wflag, sizeof(int)) != cudaSuccess || cudaMemset(wflag, 0, sizeof(int)) != cudaSuccess) {
        cudaStreamDestroy(st);
        return;
    }
    FlagScope scope(&sv->ctx->c, wflag);
    for (;;) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            // admit the head of the queue once it fits next to what is running
            sv->cv_work.wait(lk, [&] {
                return sv->stopping ||
                       (!sv->queue.empty() &&
                        (sv->in_use + sv->queue.front()->bytes <= sv->budget || sv->running == 0));
            });
            if (sv->stopping && sv->queue.empty()) break;
            if (sv->queue.empty()) continue;
            job = sv->queue.front();
            sv->queue.pop_front();
            sv->in_use += job->bytes;
            sv->running++;
            sv->peak_in_use = std::max(sv->peak_in_use, sv->in_use);
            sv->max_running = std::max(sv->max_running, sv->running);
            job->t_start = ms_since(sv);
        }
        sv->cv_work.notify_all();
        run_job(sv, st, *job);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->in_use -= job->bytes;
            sv->running--;
            job->t_done = ms_since(sv);
            job->done = true;
            job->verts.clear();
            job->verts.shrink_to_fit();
            job->tris.clear();
            job->tris.shrink_to_fit();
            job->sigma.clear();
            job->sigma.shrink_to_fit();
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
    cudaStreamDestroy(st);
    cudaFree(wflag);
}

}  // namespace
}  // namespace lsm

using namespace lsm;

extern "C" {

int lsm_server_create(lsm_ctx* ctx, int slots, int64_t hbm_budget_bytes, lsm_server** out)
{
    if (!ctx || !out || slots < 1 || slots > 64) return LSM_E_INVALID_ARG;
    *out = nullptr;
    lsm_server* sv = new (std::nothrow) lsm_server();
    if (!sv) return LSM_E_OOM;
    sv->ctx = ctx;
    if (hbm_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        cudaSetDevice(ctx->c.device);
        cudaMemGetInfo(&fr, &tot);
        hbm_budget_bytes = (int64_t)(0.8 * (double)fr);
    }
    sv->budget = hbm_budget_bytes;
    sv->t0 = Clock::now();
    for (int i = 0; i < slots; i++) sv->workers.emplace_back(worker, sv);
    {
        std::lock_guard<std::mutex> lk(ctx->c.reg_mu);
        ctx->c.servers.insert(sv);
    }
    *out = sv;
    return LSM_OK;
}

int lsm_server_submit(lsm_server* sv, const lsm_request* rq, int64_t* ticket)
{
    if (!sv || !rq || !ticket || !rq->verts || !rq->tris || rq->nv < 3 || rq->nt < 4) return LSM_E_INVALID_ARG;
    auto j = std::make_shared<Job>();
    j->verts.assign(rq->verts, rq->verts + 3 * rq->nv);
    j->tris.assign(rq->tris, rq->tris + 3 * rq->nt);
    if (rq->sigma) j->sigma.assign(rq->sigma, rq->sigma + rq->nt);
    j->rule = rq->rule.n_gl > 0 ? rq->rule : lsm_quad{4, 0};
    j->order = rq->order;
    j->tol = rq->tol;
    j->max_iter = rq->max_iter > 0 ? rq->max_iter : 20;
    j->precision = rq->precision;
    const int nq = j->rule.n_gl * j->rule.n_gl * (1 << (2 * std::max(0, j->rule.subdiv)));
    j->bytes = footprint(rq->nv, rq->nt, nq, rq->order / 2 + 2);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        j->ticket = sv->next_ticket++;
        j->t_submit = ms_since(sv);
        sv->jobs[j->ticket] = j;
        sv->queue.push_back(j);
        *ticket = j->ticket;
    }
    sv->cv_work.notify_all();
    return LSM_OK;
}

int lsm_server_poll(lsm_server* sv, int64_t ticket, int wait, lsm_result* out)
{
    if (!sv || !out) return LSM_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return LSM_E_INVALID_ARG;
    std::shared_ptr<Job> j = it->second;
    if (wait) sv->cv_done.wait(lk, [&] { return j->done; });
    if (!j->done) return LSM_PENDING;
    out->status = j->status;
    out->n_nodes = (int64_t)j->h.size();
    out->t_submit_ms = j->t_submit;
    out->t_start_ms = j->t_start;
    out->t_done_ms = j->t_done;
    out->device_bytes = j->bytes;
    out->stats = j->stats;
    out->x = j->x.empty() ? nullptr : j->x.data();
    out->h = j->h.empty() ? nullptr : j->h.data();
    out->node_status = j->node_status.empty() ? nullptr : j->node_status.data();
    out->error = j->err.c_str();
    return LSM_OK;
}

int lsm_server_cancel(lsm_server* sv, int64_t ticket)
{
    if (!sv) return LSM_E_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->jobs.find(ticket);
        if (it == sv->jobs.end()) return LSM_E_INVALID_ARG;
        auto q = std::find(sv->queue.begin(), sv->queue.end(), it->second);
        if (q == sv->queue.end()) return LSM_E_INVALID_ARG;   // already started or finished
        Job& j = **q;
        sv->queue.erase(q);
        j.status = LSM_E_CANCELLED;
        j.err = "cancelled while queued";
        j.t_start = j.t_done = ms_since(sv);
        j.done = true;
        j.verts.clear();
        j.verts.shrink_to_fit();
        j.tris.clear();
        j.tris.shrink_to_fit();
        j.sigma.clear();
        j.sigma.shrink_to_fit();
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
    return LSM_OK;
}

int lsm_server_release(lsm_server* sv, int64_t ticket)
{
    if (!sv) return LSM_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end() || !it->second->done) return LSM_E_INVALID_ARG;
    sv->jobs.erase(it);
    return LSM_OK;
}

int lsm_server_info(lsm_server* sv, lsm_server_info_t* out)
{
    if (!sv || !out) return LSM_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    out->queued = (int64_t)sv->queue.size();
    out->running = sv->running;
    out->max_running = sv->max_running;
    out->budget_bytes = sv->budget;
    out->in_use_bytes = sv->in_use;
    out->peak_in_use_bytes = sv->peak_in_use;
    out->now_ms = ms_since(sv);
    return LSM_OK;
}

int lsm_server_destroy(lsm_server* sv)
{
    if (!sv) return LSM_E_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->ctx->c.reg_mu);
        sv->ctx->c.servers.erase(sv);
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    delete sv;
    return LSM_OK;
}

}  // extern "C"
