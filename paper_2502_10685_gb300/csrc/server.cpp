// server.cpp -- stab_server_*: continuous batching of expectation and gradient
// requests.
//
// Submitted requests wait in a queue.  Planner threads admit the next one
// (the oldest, or with STAB_SERVE_SHORTEST the one with the least estimated
// work) whenever a slot and enough HBM budget are free, plan and upload
// it on a pooled context (each context has its own streams and keeps its
// device vectors between requests) and queue its kernels asynchronously;
// requests therefore join while others are running and their kernels overlap
// on the device.  A completion thread polls each request's event, copies its
// results to the host, releases its slot and budget and wakes the planners.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/stab.h"
#include "launch.h"

namespace {

struct Slot {
    stab_ctx *ctx = nullptr;
    int n = 0;
    double *d_res = nullptr;      // device: <O>
    double *d_grads = nullptr;    // device: gradient entries
    size_t grads_cap = 0;
    double *h_res = nullptr;      // pinned host copies
    double *h_grads = nullptr;
    cudaEvent_t ev = nullptr;
};

struct Req {
    int64_t id = 0;
    stab_request hdr{};
    std::vector<stab_gate> gates;
    std::vector<double> thetas;
    std::vector<stab_term> terms;
    int64_t footprint = 0;
    double work = 0.0;          // estimated work: gates x 4^n (x3 for a gradient)
    stab_result res{};
    std::vector<double> grads;
    bool done = false;
    bool admitted = false;
    Slot *slot = nullptr;
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct stab_server {
    stab_server_opts opts{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_queue, cv_done;
    std::deque<Req *> queue;
    std::unordered_map<int64_t, Req *> all;
    std::vector<Req *> active;
    std::map<int, std::vector<Slot *>> idle;
    std::vector<Slot *> slots;
    int64_t next_id = 0, submitted = 0, completed = 0, bytes_in_use = 0;
    int n_active = 0;
    bool stop = false;
    std::vector<std::thread> planners;
    std::thread completer;
};

namespace {

void complete_locked(stab_server *s, Req *r, int status) {
    r->res.status = status;
    r->res.done_s = now_s(s->t0);
    r->done = true;
    s->completed++;
}

void release_slot_locked(stab_server *s, Req *r) {
    if (r->slot) s->idle[r->slot->n].push_back(r->slot);
    r->slot = nullptr;
    if (r->admitted) {
        s->n_active--;
        s->bytes_in_use -= r->footprint;
        r->admitted = false;
    }
}

Slot *make_slot(int device, int n) {
    Slot *sl = new (std::nothrow) Slot();
    if (!sl) return nullptr;
    stab_opts o;
    stab_default_opts(&o);
    o.device = device;
    sl->n = n;
    if (stab_create(n, &o, &sl->ctx) != STAB_OK) {
        delete sl;
        return nullptr;
    }
    if (cudaMalloc(&sl->d_res, 64 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&sl->h_res, 64 * sizeof(double)) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming) != cudaSuccess) {
        stab_destroy(sl->ctx);
        if (sl->d_res) cudaFree(sl->d_res);
        if (sl->h_res) cudaFreeHost(sl->h_res);
        delete sl;
        return nullptr;
    }
    return sl;
}

void free_slot(Slot *sl) {
    if (!sl) return;
    stab_destroy(sl->ctx);
    if (sl->d_res) cudaFree(sl->d_res);
    if (sl->d_grads) cudaFree(sl->d_grads);
    if (sl->h_res) cudaFreeHost(sl->h_res);
    if (sl->h_grads) cudaFreeHost(sl->h_grads);
    if (sl->ev) cudaEventDestroy(sl->ev);
    delete sl;
}

// Plans and queues one admitted request on its slot; returns a status.
int launch_request(Req *r) {
    Slot *sl = r->slot;
    const stab_request &q = r->hdr;
    int rc = stab_load_circuit(sl->ctx, q.gates, q.m, q.thetas, q.n_params);
    if (rc == STAB_OK) rc = stab_set_observable(sl->ctx, q.obs, q.n_terms);
    if (rc != STAB_OK) return rc;
    cudaStream_t st = stab::ctx_stream(sl->ctx);
    if (q.kind == STAB_REQ_GRAD) {
        const size_t need = (size_t)(q.n_params > 0 ? q.n_params : 1);
        if (sl->grads_cap < need) {
            if (sl->d_grads) cudaFree(sl->d_grads);
            if (sl->h_grads) cudaFreeHost(sl->h_grads);
            sl->d_grads = nullptr;
            sl->h_grads = nullptr;
            sl->grads_cap = 0;
            if (cudaMalloc(&sl->d_grads, need * 8) != cudaSuccess) return STAB_E_NOMEM;
            if (cudaMallocHost(&sl->h_grads, need * 8) != cudaSuccess) return STAB_E_NOMEM;
            sl->grads_cap = need;
        }
        rc = stab_grad_async(sl->ctx, sl->d_res, sl->d_grads);
        if (rc != STAB_OK) return rc;
        if (q.n_params > 0 &&
            cudaMemcpyAsync(sl->h_grads, sl->d_grads, (size_t)q.n_params * 8,
                            cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return STAB_E_CUDA;
    } else {
        rc = stab_expect_async(sl->ctx, sl->d_res);
        if (rc != STAB_OK) return rc;
    }
    if (cudaMemcpyAsync(sl->h_res, sl->d_res, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return STAB_E_CUDA;
    if (cudaEventRecord(sl->ev, st) != cudaSuccess) return STAB_E_CUDA;
    return STAB_OK;
}

// Position in the queue of the request to admit next (caller holds s->mu).
size_t next_request_locked(const stab_server *s) {
    if (s->opts.policy != STAB_SERVE_SHORTEST) return 0;
    size_t best = 0;
    for (size_t i = 1; i < s->queue.size(); ++i)
        if (s->queue[i]->work < s->queue[best]->work) best = i;
    return best;
}

void planner_main(stab_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        size_t pick = 0;
        s->cv_queue.wait(lk, [&] {
            if (s->stop && s->queue.empty()) return true;
            if (s->queue.empty()) return false;
            pick = next_request_locked(s);
            Req *h = s->queue[pick];
            if (h->footprint > s->opts.hbm_budget) return true;   // never fits
            return s->n_active < s->opts.max_active &&
                   s->bytes_in_use + h->footprint <= s->opts.hbm_budget;
        });
        if (s->queue.empty()) {
            if (s->stop) break;
            continue;
        }
        Req *r = s->queue[pick];
        s->queue.erase(s->queue.begin() + (std::ptrdiff_t)pick);
        if (r->footprint > s->opts.hbm_budget) {
            complete_locked(s, r, STAB_E_NOMEM);
            s->cv_done.notify_all();
            continue;
        }
        r->admitted = true;
        s->n_active++;
        s->bytes_in_use += r->footprint;
        r->res.admit_s = now_s(s->t0);
        auto &pool = s->idle[r->hdr.n];
        if (!pool.empty()) {
            r->slot = pool.back();
            pool.pop_back();
        }
        lk.unlock();
        int rc = STAB_OK;
        if (!r->slot) {
            r->slot = make_slot(s->device, r->hdr.n);
            if (!r->slot) rc = STAB_E_NOMEM;
            else {
                std::lock_guard<std::mutex> g(s->mu);
                s->slots.push_back(r->slot);
            }
        }
        if (rc == STAB_OK) rc = launch_request(r);
        lk.lock();
        if (rc != STAB_OK) {
            if (r->slot) stab_synchronize(r->slot->ctx);
            release_slot_locked(s, r);
            complete_locked(s, r, rc);
            s->cv_done.notify_all();
            s->cv_queue.notify_all();
        } else {
            s->active.push_back(r);
        }
    }
}

void completer_main(stab_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        if (s->stop && s->queue.empty() && s->active.empty() && s->n_active == 0) break;
        bool any = false;
        for (size_t i = 0; i < s->active.size();) {
            Req *r = s->active[i];
            if (cudaEventQuery(r->slot->ev) != cudaSuccess) {
                ++i;
                continue;
            }
            // status word of the context (bounded device waits)
            const int st = stab_synchronize(r->slot->ctx);
            r->res.expect = r->slot->h_res[0];
            if (r->hdr.kind == STAB_REQ_GRAD && r->hdr.n_params > 0)
                r->grads.assign(r->slot->h_grads, r->slot->h_grads + r->hdr.n_params);
            release_slot_locked(s, r);
            complete_locked(s, r, st);
            s->active[i] = s->active.back();
            s->active.pop_back();
            any = true;
        }
        if (any) {
            s->cv_done.notify_all();
            s->cv_queue.notify_all();
            continue;
        }
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
    }
}

}  // namespace

extern "C" {

int64_t stab_request_footprint(const stab_request *q) {
    if (!q || q->n < 1 || q->n > STAB_MAX_QUBITS) return 0;
    const int64_t vec = (int64_t)8 << (2 * q->n);
    int64_t fp = (int64_t)q->n * vec;
    // expectation: two vector pairs of the split sweep; gradient: four (lambda, rho) pairs
    const int64_t work = vec * (q->kind == STAB_REQ_GRAD ? 8 : 4);
    if (work > fp) fp = work;
    fp += 64 * (q->m > 0 ? q->m : 0);
    if (q->kind == STAB_REQ_GRAD && q->n > stab::kMaxResidentAdjoint) {
        // per-CTA partial sums of the streamed adjoint: one per rotation and CTA
        fp += 8 * (q->m > 0 ? q->m : 0) * (int64_t)stab::adjoint_stream_blocks(q->n);
    }
    return fp;
}

int stab_server_create(const stab_server_opts *opts, stab_server **out) {
    if (!out) return STAB_E_INVAL;
    *out = nullptr;
    stab_server *s = new (std::nothrow) stab_server();
    if (!s) return STAB_E_NOMEM;
    if (opts) s->opts = *opts;
    if (s->opts.max_active <= 0) s->opts.max_active = 64;
    if (s->opts.hbm_budget <= 0) s->opts.hbm_budget = (int64_t)32 << 30;
    if (s->opts.planners <= 0) s->opts.planners = 4;
    if (s->opts.policy != STAB_SERVE_FIFO && s->opts.policy != STAB_SERVE_SHORTEST) {
        delete s;
        return STAB_E_INVAL;
    }
    int dev = s->opts.device;
    cudaError_t e = cudaSuccess;
    if (dev < 0) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        stab::record_cuda_error(e);
        delete s;
        return STAB_E_CUDA;
    }
    s->device = dev;
    s->t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < s->opts.planners; ++i) s->planners.emplace_back(planner_main, s);
    s->completer = std::thread(completer_main, s);
    *out = s;
    return STAB_OK;
}

int stab_server_submit(stab_server *s, const stab_request *req, int64_t *id) {
    if (!s || !req || !id) return STAB_E_INVAL;
    Req *r = new (std::nothrow) Req();
    if (!r) return STAB_E_NOMEM;
    r->hdr = *req;
    if (req->m > 0 && req->gates) r->gates.assign(req->gates, req->gates + req->m);
    if (req->n_params > 0 && req->thetas) r->thetas.assign(req->thetas, req->thetas + req->n_params);
    if (req->n_terms > 0 && req->obs) r->terms.assign(req->obs, req->obs + req->n_terms);
    r->hdr.gates = r->gates.empty() ? nullptr : r->gates.data();
    r->hdr.thetas = r->thetas.empty() ? nullptr : r->thetas.data();
    r->hdr.obs = r->terms.empty() ? nullptr : r->terms.data();
    r->footprint = stab_request_footprint(req);
    if (req->n >= 1 && req->n <= STAB_MAX_QUBITS)
        r->work = (double)(req->m > 0 ? req->m : 1) * (double)(1ull << (2 * req->n)) *
                  (req->kind == STAB_REQ_GRAD ? 3.0 : 1.0);
    r->res.n_params = (int32_t)req->n_params;
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->res.submit_s = now_s(s->t0);
    s->all[r->id] = r;
    s->submitted++;
    if (req->n < 1 || req->n > STAB_MAX_QUBITS ||
        (req->kind != STAB_REQ_EXPECT && req->kind != STAB_REQ_GRAD)) {
        complete_locked(s, r, req->n < 1 || req->n > STAB_MAX_QUBITS ? STAB_E_RANGE : STAB_E_INVAL);
        s->cv_done.notify_all();
    } else {
        s->queue.push_back(r);
        s->cv_queue.notify_one();
    }
    *id = r->id;
    return STAB_OK;
}

int stab_server_wait(stab_server *s, int64_t id, double timeout_s, stab_result *out,
                     double *grads) {
    if (!s) return STAB_E_INVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return STAB_E_INVAL;
    Req *r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_s < 0) {
        s->cv_done.wait(lk, pred);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        return STAB_E_TIMEOUT;
    }
    if (out) *out = r->res;
    if (grads && !r->grads.empty()) std::memcpy(grads, r->grads.data(), r->grads.size() * 8);
    // the results are handed out: the request is released
    s->all.erase(it);
    delete r;
    return STAB_OK;
}

int stab_server_poll(stab_server *s, int64_t id, int32_t *done) {
    if (!s || !done) return STAB_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return STAB_E_INVAL;
    *done = it->second->done ? 1 : 0;
    return STAB_OK;
}

int stab_server_stats(stab_server *s, int64_t *submitted, int64_t *completed, int64_t *active,
                      int64_t *bytes_in_use) {
    if (!s) return STAB_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (submitted) *submitted = s->submitted;
    if (completed) *completed = s->completed;
    if (active) *active = s->n_active;
    if (bytes_in_use) *bytes_in_use = s->bytes_in_use;
    return STAB_OK;
}

int stab_server_destroy(stab_server *s) {
    if (!s) return STAB_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_queue.notify_all();
    for (auto &t : s->planners) t.join();
    s->completer.join();
    cudaSetDevice(s->device);
    for (Slot *sl : s->slots) free_slot(sl);
    for (auto &kv : s->all) delete kv.second;
    delete s;
    return STAB_OK;
}

}  // extern "C"
