// liblbib serving engine (include/lbib.h, lbib_serve_*): runs submitted
// lattice-Boltzmann / immersed-boundary requests to completion on one GPU.
//
// A worker thread admits queued requests in arrival order while their
// estimated device memory fits the budget, creates their contexts, and
// advances every admitted run together as one batch (lbib_batch_*), a chunk
// of steps at a time.  A chunk ends when the run with the fewest remaining
// steps finishes; finished runs leave the batch (their contexts stay
// resident until the caller takes them), new arrivals join, and the batch is
// rebuilt: continuous batching.  A chunk with a single run advances it with
// lbib_step.  The plain mode runs one request at a time with lbib_step, in
// arrival order, for comparison.
//
// Built on the public C ABI only.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lbib.h"

namespace {

using Clock = std::chrono::steady_clock;

struct ReqBody {
    std::vector<double> verts;
    std::vector<int> tris;
    lbib_body_params bp;
};

struct Request {
    lbib_params p{};
    long long nsteps = 0;
    int init = 0;
    std::vector<ReqBody> bodies;
    // run state
    long long id = 0;
    void *ctx = nullptr;
    long long remaining = 0;
    size_t bytes = 0;
    int state = LBIB_REQ_QUEUED;
    int err = 0;
    std::string msg;  // why a failed run failed
    Clock::time_point t_submit, t_admit, t_done;
};

struct Server {
    lbib_serve_params sp{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;      // submitted, not admitted
    std::vector<Request *> active;    // admitted, running
    std::map<long long, Request *> all;
    long long next_id = 1;
    size_t bytes_in_use = 0, peak_bytes = 0;
    double cell_updates = 0.0, busy_s = 0.0;
    long long runs_done = 0, runs_failed = 0, chunks = 0, rebuilds = 0;
    bool stop = false;
    std::thread worker;
    cudaStream_t stream = nullptr;
};

size_t estimate_bytes(const Request &r) {
    const size_t ncell = (size_t)r.p.nx * r.p.ny * r.p.nz;
    const size_t stride = (ncell + 63) / 64 * 64;
    const size_t elem = r.p.precision == LBIB_FP64 ? 8 : r.p.precision == LBIB_FP32 ? 4 : 2;
    const size_t relem = r.p.precision == LBIB_FP64 ? 8 : 4;
    size_t b = stride * (2 * 19 * elem + 11 * relem) + ncell / 128 + (1 << 16);
    for (const ReqBody &rb : r.bodies) {
        const size_t nv = rb.verts.size() / 3, nt = rb.tris.size() / 3;
        b += nv * (27 * (4 + relem) + 12 * 8 + 64) + nt * (24 * relem + 128) + (1 << 16);
    }
    return b;
}

double seconds(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double>(b - a).count();
}

// Creates the context of an admitted request; returns an lbib code.
int start_request(Server *s, Request *r) {
    lbib_params p = r->p;
    p.stream = s->stream;
    p.alloc = nullptr;
    p.free = nullptr;
    int rc = lbib_create(&p, &r->ctx);
    if (rc) return rc;
    if (r->init == 1) {
        // the exact Couette profile between the z walls (x velocity linear in z)
        rc = lbib_set_shear_fields(r->ctx, p.wall_u[4][0], p.wall_u[5][0]);
        if (rc == LBIB_OK) rc = lbib_sync(r->ctx);
        if (rc) return rc;
    }
    for (ReqBody &rb : r->bodies) {
        rc = lbib_add_body(r->ctx, rb.verts.data(), (int)(rb.verts.size() / 3), rb.tris.data(),
                           (int)(rb.tris.size() / 3), &rb.bp, nullptr);
        if (rc) return rc;
        std::vector<double>().swap(rb.verts);
        std::vector<int>().swap(rb.tris);
    }
    return LBIB_OK;
}

void finish(Server *s, Request *r, int err, const char *why = nullptr) {
    r->t_done = Clock::now();
    r->err = err;
    r->state = err ? LBIB_REQ_FAILED : LBIB_REQ_DONE;
    if (err) {
        if (why)
            r->msg = why;
        else if (r->ctx)
            r->msg = lbib_last_error(r->ctx);
        else
            r->msg = lbib_last_error(nullptr);
        if (r->ctx) lbib_destroy(r->ctx);
        r->ctx = nullptr;
        s->bytes_in_use -= r->bytes;
        r->bytes = 0;
        ++s->runs_failed;
    } else {
        ++s->runs_done;
    }
}

void worker_loop(Server *s) {
    cudaSetDevice(s->device);
    void *batch = nullptr;
    bool stale = true;
    std::vector<Request *> members;
    for (;;) {
        std::vector<Request *> admitted;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // admission in arrival order while the memory estimate fits
            while (!s->queue.empty()) {
                Request *r = s->queue.front();
                const size_t need = estimate_bytes(*r);
                const int cap = s->sp.mode == LBIB_SERVE_PLAIN ? 1 : s->sp.max_active;
                if (need > s->sp.hbm_budget) {  // can never fit
                    s->queue.pop_front();
                    r->t_admit = Clock::now();
                    finish(s, r, LBIB_ENOMEM, "the run's memory estimate exceeds the budget");
                    s->cv_done.notify_all();
                    continue;
                }
                if ((int)(s->active.size() + admitted.size()) >= cap) break;
                if (s->bytes_in_use + need > s->sp.hbm_budget) break;
                s->queue.pop_front();
                r->bytes = need;
                s->bytes_in_use += need;
                s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_use);
                r->state = LBIB_REQ_RUNNING;
                r->t_admit = Clock::now();
                admitted.push_back(r);
            }
            if (admitted.empty() && s->active.empty()) {
                if (s->stop) break;
                s->cv_work.wait(lk);
                continue;
            }
        }
        for (Request *r : admitted) {
            int rc = start_request(s, r);
            std::lock_guard<std::mutex> lk(s->mu);
            if (rc) {
                finish(s, r, rc);
                s->cv_done.notify_all();
            } else {
                r->remaining = r->nsteps;
                s->active.push_back(r);
                stale = true;
            }
        }
        std::vector<Request *> act;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            act = s->active;
        }
        if (act.empty()) continue;
        if (s->sp.mode == LBIB_SERVE_BATCHED && s->sp.batch_cells > 0 && act.size() > 1) {
            // up to batch_cells lattice cells of runs (at least one run),
            // the runs with the least remaining cell updates first or the
            // earliest submitted first; the others stay resident and wait
            if (s->sp.batch_order == LBIB_SERVE_OLDEST)
                std::stable_sort(act.begin(), act.end(), [](const Request *a, const Request *b) { return a->id < b->id; });
            else
                std::stable_sort(act.begin(), act.end(), [](const Request *a, const Request *b) {
                    const double wa = (double)a->remaining * a->p.nx * a->p.ny * a->p.nz;
                    const double wb = (double)b->remaining * b->p.nx * b->p.ny * b->p.nz;
                    return wa < wb;
                });
            long long cells = 0;
            size_t k = 0;
            for (; k < act.size(); ++k) {
                const long long c = (long long)act[k]->p.nx * act[k]->p.ny * act[k]->p.nz;
                if (k > 0 && cells + c > s->sp.batch_cells) break;
                cells += c;
            }
            act.resize(k);
        }
        long long chunk = s->sp.chunk_steps > 0 ? s->sp.chunk_steps : 500;
        for (Request *r : act) chunk = std::min(chunk, r->remaining);
        const auto t_a = Clock::now();
        int brc = LBIB_OK;
        bool advanced = false;  // the chunk's steps were enqueued for every run
        if (s->sp.mode == LBIB_SERVE_PLAIN || act.size() == 1) {
            // one run: its own step (the IB stage beside the far-field
            // sweep, the context's sweep shape), as in plain mode; a batch
            // that holds the context is rebuilt before it is used again
            brc = lbib_step(act[0]->ctx, (int)chunk);
            advanced = brc == LBIB_OK;
            if (!brc) brc = lbib_sync(act[0]->ctx);
            stale = true;
        } else {
            if (stale || act != members) {
                if (batch) lbib_batch_destroy(batch);
                batch = nullptr;
                std::vector<void *> ctxs;
                for (Request *r : act) ctxs.push_back(r->ctx);
                brc = lbib_batch_create(ctxs.data(), (int)ctxs.size(), s->stream, &batch);
                members = act;
                stale = false;
                ++s->rebuilds;
            }
            if (!brc) {
                brc = lbib_batch_step(batch, (int)chunk);
                advanced = brc == LBIB_OK;
            }
            if (!brc) brc = lbib_batch_sync(batch);
        }
        const auto t_b = Clock::now();
        std::lock_guard<std::mutex> lk(s->mu);
        s->busy_s += seconds(t_a, t_b);
        ++s->chunks;
        std::vector<Request *> keep;
        for (Request *r : s->active)  // runs that waited this chunk
            if (std::find(act.begin(), act.end(), r) == act.end()) keep.push_back(r);
        const size_t waited = keep.size();
        for (Request *r : act) {
            int rc = LBIB_OK;
            if (brc) rc = lbib_sync(r->ctx);  // which run failed
            if (rc) {
                finish(s, r, rc);
                stale = true;
                continue;
            }
            if (advanced) {
                r->remaining -= chunk;
                s->cell_updates += (double)chunk * r->p.nx * r->p.ny * r->p.nz;
            }
            if (r->remaining <= 0) {
                // a finished run passes the divergence watchdog once more on
                // its final state (its cadence may not have fallen on it)
                finish(s, r, lbib_check(r->ctx));
                stale = true;
            } else {
                keep.push_back(r);
            }
        }
        if (brc && keep.size() - waited == act.size()) {
            // a batch-level failure no single context reports: fail them all
            const std::string why = batch ? lbib_batch_last_error(batch) : lbib_batch_last_error(nullptr);
            for (size_t k = waited; k < keep.size(); ++k) finish(s, keep[k], brc, why.c_str());
            keep.resize(waited);
            stale = true;
        }
        s->active = keep;
        s->cv_done.notify_all();
    }
    if (batch) lbib_batch_destroy(batch);
}

Server *as_server(void *h) { return static_cast<Server *>(h); }

}  // namespace

extern "C" {

int lbib_request_create(const lbib_params *p, long long nsteps, int init, void **req) {
    if (!p || !req || nsteps < 0 || init < 0 || init > 1) return LBIB_EINVAL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || !(p->tau > 0.5)) return LBIB_EINVAL;
    Request *r = new Request();
    r->p = *p;
    r->nsteps = nsteps;
    r->init = init;
    *req = r;
    return LBIB_OK;
}

int lbib_request_add_body(void *req, const double *verts, int nv, const int *tris, int nt,
                          const lbib_body_params *bp) {
    Request *r = static_cast<Request *>(req);
    if (!r || !verts || !tris || !bp || nv < 4 || nt < 4 || r->state != LBIB_REQ_QUEUED || r->id) return LBIB_EINVAL;
    ReqBody b;
    b.verts.assign(verts, verts + 3 * (size_t)nv);
    b.tris.assign(tris, tris + 3 * (size_t)nt);
    b.bp = *bp;
    r->bodies.push_back(std::move(b));
    return LBIB_OK;
}

void lbib_request_destroy(void *req) {
    Request *r = static_cast<Request *>(req);
    if (r && !r->id) delete r;
}

int lbib_serve_create(const lbib_serve_params *sp, void **out) {
    if (!sp || !out || sp->hbm_budget == 0 || sp->max_active < 1 ||
        (sp->mode != LBIB_SERVE_BATCHED && sp->mode != LBIB_SERVE_PLAIN) ||
        (sp->batch_order != LBIB_SERVE_SHORTEST && sp->batch_order != LBIB_SERVE_OLDEST))
        return LBIB_EINVAL;
    Server *s = new Server();
    s->sp = *sp;
    s->t0 = Clock::now();
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return LBIB_ECUDA;
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return LBIB_OK;
}

int lbib_serve_submit(void *h, void *req, long long *id) {
    Server *s = as_server(h);
    Request *r = static_cast<Request *>(req);
    if (!s || !r || r->id) return LBIB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    r->state = LBIB_REQ_QUEUED;
    s->all[r->id] = r;
    s->queue.push_back(r);
    if (id) *id = r->id;
    s->cv_work.notify_one();
    return LBIB_OK;
}

int lbib_serve_wait(void *h, long long id, double timeout_s, int *state) {
    Server *s = as_server(h);
    if (!s) return LBIB_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return LBIB_EINVAL;
    Request *r = it->second;
    auto done = [&] { return r->state == LBIB_REQ_DONE || r->state == LBIB_REQ_FAILED; };
    if (timeout_s < 0)
        s->cv_done.wait(lk, done);
    else
        s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
    if (state) *state = r->state;
    return done() ? (r->state == LBIB_REQ_FAILED ? r->err : LBIB_OK) : LBIB_ETIMEOUT;
}

int lbib_serve_take(void *h, long long id, void **ctx, lbib_serve_times *t) {
    Server *s = as_server(h);
    if (!s || !ctx) return LBIB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return LBIB_EINVAL;
    Request *r = it->second;
    if (r->state != LBIB_REQ_DONE && r->state != LBIB_REQ_FAILED) return LBIB_EINVAL;
    if (t) {
        t->queued_s = seconds(r->t_submit, r->t_admit);
        t->latency_s = seconds(r->t_submit, r->t_done);
        t->submit_s = seconds(s->t0, r->t_submit);
        t->done_s = seconds(s->t0, r->t_done);
        std::snprintf(t->error, sizeof(t->error), "%s", r->msg.c_str());
    }
    const int err = r->state == LBIB_REQ_FAILED ? r->err : LBIB_OK;
    *ctx = r->ctx;
    s->bytes_in_use -= r->bytes;
    s->all.erase(it);
    delete r;
    s->cv_work.notify_one();  // memory freed up for admission
    return err;
}

int lbib_serve_stats(void *h, lbib_serve_summary *out) {
    Server *s = as_server(h);
    if (!s || !out) return LBIB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->runs_done = s->runs_done;
    out->runs_failed = s->runs_failed;
    out->queued = (long long)s->queue.size();
    out->active = (long long)s->active.size();
    out->chunks = s->chunks;
    out->rebuilds = s->rebuilds;
    out->cell_updates = s->cell_updates;
    out->busy_s = s->busy_s;
    out->bytes_in_use = s->bytes_in_use;
    out->peak_bytes = s->peak_bytes;
    return LBIB_OK;
}

void lbib_serve_destroy(void *h) {
    Server *s = as_server(h);
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // queued requests are dropped; running ones finish their runs first
        for (Request *r : s->queue) r->state = LBIB_REQ_FAILED;
        s->queue.clear();
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->all) {
        if (kv.second->ctx) lbib_destroy(kv.second->ctx);
        delete kv.second;
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
