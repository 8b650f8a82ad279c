// Request server: assemble-and-solve requests of different meshes, deltas,
// strategies and precisions, served continuously on one GPU.
//
//  * Workers: each worker thread owns a CUDA stream and takes requests one at
//    a time; up to `workers` requests are on the device at once and their
//    kernels overlap.  A request that arrives while others run starts as soon
//    as a worker is free and its footprint fits.
//  * Admission: a request's device footprint is estimated from its size
//    (pairs ~ outer elements x the ball's element count); the head of the
//    queue starts only while the running requests' estimates plus the
//    resident cache stay within the budget.  Least recently used cache
//    entries that no running request holds are evicted to make room.
//  * Residency: the mesh, the pair list and the sparsity pattern of a
//    (box, delta) key stay on the device between requests.
//  * Memory: stream-ordered allocation (cudaMallocAsync / cudaFreeAsync on
//    the worker's stream), so no request's allocations synchronise another's
//    work.
// Every kernel of a request is the single-problem code path, so a request's
// result is the same whether it runs alone or among others.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "nl_internal.h"

namespace {

__global__ void k_quadratic_g(const double4 *__restrict__ v, int64_t nv, double *g)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv) {
        const double4 p = v[i];
        g[i] = (p.x * p.x + p.y * p.y) + p.z * p.z;
    }
}

struct Worker;

struct CacheEntry {
    double lo, hi, olo, ohi, delta, jitter;
    uint64_t jitter_seed;
    int cells;
    nl_mesh *mesh = nullptr;
    nl_pairs *pairs = nullptr;
    int64_t bytes = 0;
    int refs = 0;
    uint64_t last_use = 0;
};

struct Job {
    uint64_t ticket = 0;
    nl_request req{};
    int64_t est = 0;
    nl_result res{};
    std::vector<double> u;
};

void *worker_alloc(size_t n, void *ctx);
void worker_free(void *p, void *ctx);

}  // namespace

struct nl_server {
    nl_server_opts opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> queue;
    std::map<uint64_t, Job *> jobs;
    std::vector<CacheEntry *> cache;
    std::vector<Worker *> workers;
    int64_t running_bytes = 0, cache_bytes = 0;
    int running = 0;
    uint64_t next_ticket = 1, use_clock = 0;
    bool stop = false;
    std::chrono::steady_clock::time_point t0;
    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

struct Worker {
    nl_server *srv = nullptr;
    cudaStream_t s = nullptr;
    nl_device dev{};
    std::thread th;
};

void *worker_alloc(size_t n, void *ctx)
{
    Worker *w = static_cast<Worker *>(ctx);
    void *p = nullptr;
    if (cudaMallocAsync(&p, n, w->s) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

void worker_free(void *p, void *ctx)
{
    Worker *w = static_cast<Worker *>(ctx);
    cudaFreeAsync(p, w->s);
}

// Device bytes a request may hold while it runs (an estimate for admission).
int64_t estimate_bytes(const nl_request &r)
{
    const double h = (r.hi - r.lo) / r.cells;
    const double ratio = r.delta / h;
    const double n_omega = (r.omega_hi - r.omega_lo) / h;
    const double n_outer = 6.0 * n_omega * n_omega * n_omega;
    const double pairs = n_outer * 6.0 * (4.0 * M_PI / 3.0) * pow(ratio + 1.0, 3.0);
    const double nt = 6.0 * (double)r.cells * r.cells * r.cells;
    const double sz = r.assemble.precision == NL_FP32_COMP ? 4.0 : 8.0;
    const double units = std::min(4.0 * pairs, (double)(int64_t(1) << 25));
    const double b = pairs * (12.0 + 10.0 * sz + 24.0) + units * (21.0 + 16.0 * sz) + nt * 400.0;
    return (int64_t)b;
}

int64_t resident_bytes(const nl_pairs *P)
{
    const nl_mesh *m = P->mesh;
    return (int64_t)(P->npairs * 12 + P->nnz * 16 + P->nnz_a * 12 + m->nv * 120 + m->nt * 200 + m->n_outer * 200);
}

bool same_key(const CacheEntry *e, const nl_request &r)
{
    return e->cells == r.cells && e->lo == r.lo && e->hi == r.hi && e->olo == r.omega_lo && e->ohi == r.omega_hi &&
           e->jitter == r.jitter_frac && e->jitter_seed == r.jitter_seed &&
           e->delta == r.delta;
}

void destroy_entry(CacheEntry *e)
{
    if (e->pairs) nl_pairs_destroy(e->pairs);
    if (e->mesh) nl_mesh_destroy(e->mesh);
    delete e;
}

// Evict unreferenced entries, least recently used first, until `need` more
// bytes fit.  Called with the lock held.
void evict_for(nl_server *S, int64_t need)
{
    while (S->running_bytes + S->cache_bytes + need > S->opts.budget_bytes) {
        CacheEntry *victim = nullptr;
        for (CacheEntry *e : S->cache)
            if (e->refs == 0 && (!victim || e->last_use < victim->last_use)) victim = e;
        if (!victim) return;
        S->cache.erase(std::find(S->cache.begin(), S->cache.end(), victim));
        S->cache_bytes -= victim->bytes;
        destroy_entry(victim);
    }
}

void run_job(Worker *w, Job *J)
{
    nl_server *S = w->srv;
    const nl_request &r = J->req;
    CacheEntry *ent = nullptr;
    nl_system *sys = nullptr;
    double *g = nullptr, *ud = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    try {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (CacheEntry *e : S->cache)
                if (same_key(e, r)) { ent = e; break; }
            if (ent) { ent->refs++; ent->last_use = ++S->use_clock; J->res.cache_hit = 1; }
        }
        if (!ent) {
            CacheEntry *e = new CacheEntry();
            e->lo = r.lo; e->hi = r.hi; e->olo = r.omega_lo; e->ohi = r.omega_hi; e->delta = r.delta;
            e->cells = r.cells;
            e->jitter = r.jitter_frac;
            e->jitter_seed = r.jitter_seed;
            nl_status st = nl_mesh_create_box(&w->dev, r.lo, r.hi, r.cells, r.omega_lo, r.omega_hi, r.jitter_frac,
                                              r.jitter_seed, &e->mesh);
            if (st == NL_OK) st = nl_pairs_build(e->mesh, r.delta, &e->pairs);
            if (st != NL_OK) {
                snprintf(J->res.message, sizeof(J->res.message), "%s", nl_last_error());
                destroy_entry(e);
                throw NlError{st};
            }
            e->bytes = resident_bytes(e->pairs);
            std::lock_guard<std::mutex> lk(S->mu);
            e->refs = 1;
            e->last_use = ++S->use_clock;
            S->cache.push_back(e);
            S->cache_bytes += e->bytes;
            ent = e;
        }
        nl_pairs *P = ent->pairs;
        nl_mesh *m = P->mesh;
        J->res.n_pairs = P->npairs;
        J->res.n_free = m->n_free;
        J->res.n_vert = m->nv;
        for (auto &e : ev) NL_CUDA(cudaEventCreate(&e));
        NL_CUDA(cudaEventRecord(ev[0], w->s));
        nl_assemble_opts ao = r.assemble;
        if (r.g_quadratic) {
            g = static_cast<double *>(worker_alloc(sizeof(double) * m->nv, w));
            if (!g) { nl_set_error("device allocation failed"); throw NlError{NL_ENOMEM}; }
            { k_quadratic_g<<<(unsigned)nl_cdiv<int64_t>(m->nv, 256), 256, 0, w->s>>>(m->verts, m->nv, g); nl_count_launch(); }
            NL_CHECK_LAUNCH();
            ao.g_nodal = g;
            ao.g_where = NL_DEVICE;
        } else {
            ao.g_nodal = nullptr;
        }
        nl_status st = nl_assemble_on(P, &ao, &w->dev, &sys);
        if (st != NL_OK) {
            snprintf(J->res.message, sizeof(J->res.message), "%s", nl_last_error());
            throw NlError{st};
        }
        NL_CUDA(cudaEventRecord(ev[1], w->s));
        ud = static_cast<double *>(worker_alloc(sizeof(double) * m->nv, w));
        if (!ud) { nl_set_error("device allocation failed"); throw NlError{NL_ENOMEM}; }
        nl_solve_info si{};
        st = nl_solve_impl(sys, &r.solve, ud, NL_DEVICE, &si);
        if (st != NL_OK && st != NL_ENOTCONV) {
            snprintf(J->res.message, sizeof(J->res.message), "%s", nl_last_error());
            throw NlError{st};
        }
        J->res.status = st;
        J->res.iterations = si.iterations;
        J->res.refinements = si.refinements;
        J->res.rel_residual = si.rel_residual;
        NL_CUDA(cudaEventRecord(ev[2], w->s));
        J->u.resize(m->nv);
        NL_CUDA(cudaMemcpyAsync(J->u.data(), ud, sizeof(double) * m->nv, cudaMemcpyDeviceToHost, w->s));
        NL_CUDA(cudaStreamSynchronize(w->s));
        float a = 0.f, b = 0.f;
        NL_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
        NL_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
        J->res.assemble_ms = a;
        J->res.solve_ms = b;
    } catch (NlError &e) {
        J->res.status = e.st;
        if (!J->res.message[0]) snprintf(J->res.message, sizeof(J->res.message), "%s", nl_last_error());
    }
    if (sys) nl_system_destroy(sys);
    if (g) worker_free(g, w);
    if (ud) worker_free(ud, w);
    cudaStreamSynchronize(w->s);
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    std::lock_guard<std::mutex> lk(S->mu);
    if (ent) {
        ent->refs--;
        ent->last_use = ++S->use_clock;
        if (!S->opts.cache && ent->refs == 0) {
            S->cache.erase(std::find(S->cache.begin(), S->cache.end(), ent));
            S->cache_bytes -= ent->bytes;
            destroy_entry(ent);
        }
    }
}

void worker_main(Worker *w)
{
    nl_server *S = w->srv;
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        Job *J = nullptr;
        while (!S->stop) {
            if (!S->queue.empty()) {
                Job *head = S->queue.front();
                if (head->est > S->opts.budget_bytes) {
                    // can never fit: fail it
                    S->queue.pop_front();
                    head->res.status = NL_ENOMEM;
                    snprintf(head->res.message, sizeof(head->res.message),
                             "estimated footprint %lld bytes exceeds the budget", (long long)head->est);
                    head->res.t_start = head->res.t_done = S->now();
                    head->res.state = NL_REQ_DONE;
                    S->cv_done.notify_all();
                    continue;
                }
                evict_for(S, head->est);
                if (S->running == 0 || S->running_bytes + S->cache_bytes + head->est <= S->opts.budget_bytes) {
                    J = head;
                    S->queue.pop_front();
                    break;
                }
            }
            S->cv_work.wait(lk);
        }
        if (!J) return;
        S->running++;
        S->running_bytes += J->est;
        J->res.state = NL_REQ_RUNNING;
        J->res.t_start = S->now();
        J->res.queue_depth_at_start = (int)S->queue.size();
        lk.unlock();
        run_job(w, J);
        lk.lock();
        S->running--;
        S->running_bytes -= J->est;
        J->res.t_done = S->now();
        J->res.state = NL_REQ_DONE;
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace

extern "C" nl_status nl_server_create(const nl_server_opts *opts, nl_server **out)
{
    nl_clear_error();
    if (!opts || !out) { nl_set_error("NULL argument"); return NL_EINVAL; }
    *out = nullptr;
    if (opts->workers < 1 || opts->workers > 16 || opts->budget_bytes <= 0 || opts->queue_capacity < 1) {
        nl_set_error("bad server options (workers 1..16, budget > 0, queue capacity >= 1)");
        return NL_EINVAL;
    }
    nl_server *S = new nl_server();
    S->opts = *opts;
    S->t0 = std::chrono::steady_clock::now();
    try {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            (void)cudaGetLastError();
            nl_set_error("no CUDA device available");
            throw NlError{NL_ECUDA};
        }
        NL_CUDA(cudaGetDevice(&S->device));
        // keep freed blocks in this process's default pool between requests
        cudaMemPool_t pool;
        NL_CUDA(cudaDeviceGetDefaultMemPool(&pool, S->device));
        uint64_t thr = UINT64_MAX;
        NL_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        for (int i = 0; i < opts->workers; ++i) {
            Worker *w = new Worker();
            S->workers.push_back(w);    // owned by the server before anything can fail
            w->srv = S;
            NL_CUDA(cudaStreamCreateWithFlags(&w->s, cudaStreamNonBlocking));
            w->dev.alloc = worker_alloc;
            w->dev.free = worker_free;
            w->dev.ctx = w;
            w->dev.stream = w->s;
        }
        for (Worker *w : S->workers) w->th = std::thread(worker_main, w);
    } catch (NlError &e) {
        for (Worker *w : S->workers) {
            if (w->s) cudaStreamDestroy(w->s);
            delete w;
        }
        delete S;
        return e.st;
    }
    *out = S;
    return NL_OK;
}

extern "C" nl_status nl_server_submit(nl_server *S, const nl_request *req, uint64_t *ticket)
{
    nl_clear_error();
    if (!S || !req || !ticket) { nl_set_error("NULL argument"); return NL_EINVAL; }
    if (req->cells < 1 || !(req->delta > 0.0) || !isfinite(req->delta) || !(req->hi > req->lo)) {
        nl_set_error("bad request geometry");
        return NL_EINVAL;
    }
    if (req->assemble.g_nodal) { nl_set_error("requests carry g as g_quadratic, not g_nodal"); return NL_EINVAL; }
    if (req->assemble.f_nodal) { nl_set_error("requests carry a constant f (f_nodal must be NULL)"); return NL_EINVAL; }
    if (req->assemble.kernel_poly) { nl_set_error("a kernel shape (kernel_poly) runs through nl_assemble only"); return NL_EINVAL; }
    if (nl_status st = nl_check_assemble_opts(&req->assemble)) return st;
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->queue.size() >= S->opts.queue_capacity) { nl_set_error("queue full"); return NL_EBUSY; }
    Job *J = new Job();
    J->ticket = S->next_ticket++;
    J->req = *req;
    J->est = estimate_bytes(*req);
    J->res.state = NL_REQ_QUEUED;
    J->res.t_submit = S->now();
    J->res.est_bytes = J->est;
    S->jobs[J->ticket] = J;
    S->queue.push_back(J);
    *ticket = J->ticket;
    S->cv_work.notify_one();
    return NL_OK;
}

extern "C" nl_status nl_server_poll(nl_server *S, uint64_t ticket, nl_result *res)
{
    nl_clear_error();
    if (!S || !res) { nl_set_error("NULL argument"); return NL_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) { nl_set_error("unknown ticket"); return NL_EINVAL; }
    *res = it->second->res;
    return NL_OK;
}

extern "C" nl_status nl_server_wait(nl_server *S, uint64_t ticket, double timeout_s, nl_result *res, double *u_out,
                                    int64_t n_u)
{
    nl_clear_error();
    if (!S) { nl_set_error("NULL argument"); return NL_EINVAL; }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) { nl_set_error("unknown ticket"); return NL_EINVAL; }
    Job *J = it->second;
    auto done = [&] { return J->res.state == NL_REQ_DONE; };
    if (timeout_s > 0.0) {
        if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
            nl_set_error("request %llu not done after %.3f s", (unsigned long long)ticket, timeout_s);
            if (res) *res = J->res;
            return NL_ETIMEOUT;
        }
    } else {
        S->cv_done.wait(lk, done);
    }
    if (res) *res = J->res;
    if (u_out) {
        if (n_u < (int64_t)J->u.size()) { nl_set_error("u_out holds %lld values, %zu needed", (long long)n_u, J->u.size()); return NL_EINVAL; }
        memcpy(u_out, J->u.data(), sizeof(double) * J->u.size());
    }
    return NL_OK;
}

extern "C" nl_status nl_server_release(nl_server *S, uint64_t ticket)
{
    nl_clear_error();
    if (!S) { nl_set_error("NULL argument"); return NL_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) { nl_set_error("unknown ticket"); return NL_EINVAL; }
    if (it->second->res.state != NL_REQ_DONE) { nl_set_error("request still in flight"); return NL_EBUSY; }
    delete it->second;
    S->jobs.erase(it);
    return NL_OK;
}

extern "C" nl_status nl_server_get_load(nl_server *S, nl_server_load *out)
{
    nl_clear_error();
    if (!S || !out) { nl_set_error("NULL argument"); return NL_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    out->queued = (int)S->queue.size();
    out->running = S->running;
    out->cache_entries = (int)S->cache.size();
    out->cache_bytes = S->cache_bytes;
    out->running_bytes = S->running_bytes;
    return NL_OK;
}

extern "C" void nl_server_destroy(nl_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // requests that never started are dropped
        for (Job *J : S->queue) {
            J->res.state = NL_REQ_DONE;
            J->res.status = NL_EINVAL;
        }
        S->queue.clear();
    }
    S->cv_work.notify_all();
    for (Worker *w : S->workers)
        if (w->th.joinable()) w->th.join();
    for (CacheEntry *e : S->cache) destroy_entry(e);
    for (Worker *w : S->workers) {
        cudaStreamSynchronize(w->s);
        cudaStreamDestroy(w->s);
        delete w;
    }
    for (auto &kv : S->jobs) delete kv.second;
    delete S;
}
