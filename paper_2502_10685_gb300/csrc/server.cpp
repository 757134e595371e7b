// server.cpp -- stab_server_*: continuous batching of expectation and gradient
// requests.
//
// Submitted requests wait in a queue.  Planner threads admit the next one
// (the oldest, or with STAB_SERVE_SHORTEST the one with the least estimated
// work unless the oldest has waited longer than the aging bound) whenever a
// slot and enough HBM budget are free.  Two engines then run it:
//
//  * the iteration engine (STAB_SERVE_ITERATE, requests of n <= iter_max_n): the
//    planner thread plans the request on the host; the engine thread uploads
//    it into one device block and, once per iteration, launches one
//    persistent k_serve kernel that advances every admitted request by a
//    slice of its instruction streams (a fixed number of chunks per n).  The
//    requests' vectors stay in their device blocks between iterations, new
//    requests join at the next iteration, finished ones leave after the
//    launch that finished them.  Two iterations are in flight at a time, so
//    the host prepares the next launch while the GPU runs the current one.
//  * the context engine (every request with STAB_SERVE_CONTEXTS, and larger
//    requests with ITERATE): the request runs on a pooled context with its own
//    streams (the vectors of a large request fill the GPU by themselves);
//    its kernels overlap on the device with every other request's.  A
//    completion thread polls each request's event.
//
// Device memory comes from the allocator hooks of the options (else
// cudaMallocAsync / cudaFreeAsync on the engine's or context's stream) and is
// given back only after the work that used it has completed.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
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
#include "planner.h"

using namespace stab;

namespace {

constexpr int kInFlight = 2;          // iterations queued on the GPU at once
constexpr int kTableSlots = kInFlight + 1;
constexpr int kDefaultIterChunks = 32;   // a Poisson trace of n = 4..8 requests, two runs each:
                                         // 16 / 32 / 64 / 128 chunks gave 990 / 1,079 / 1,044 /
                                         // 993 circuits/s and p99 200 / 183 / 207 / 224 ms
constexpr int kDefaultIterSmemKb = 32;
// Requests above this size go to contexts by default: one CTA per vector
// leaves a 4^7 or 4^8 vector latency-bound, while a context streams it over
// the whole GPU (a Poisson trace of n = 4..8 requests: 1,068 circuits/s with
// n <= 6 in the iteration engine, 380 with n <= 8, 604 with contexts only).
constexpr int kDefaultIterMaxN = 6;
constexpr double kDefaultAgingS = 4.0;
constexpr double kDefaultIterSliceUs = 400.0;
constexpr int kCostClasses = (kServeMaxQubits + 1) * 3 * 2;

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Hooks {
    stab_alloc_fn alloc = nullptr;
    stab_free_fn free = nullptr;
    void *user = nullptr;
    void *get(size_t bytes, cudaStream_t st) const {
        void *p = nullptr;
        if (alloc) return alloc(bytes, (void *)st, user);
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void put(void *p, size_t bytes, cudaStream_t st) const {
        if (!p) return;
        if (free) free(p, bytes, (void *)st, user);
        else cudaFreeAsync(p, st);
    }
};

// Pinned host blocks, reused across requests (cudaMallocHost is slow).
class PinnedPool {
public:
    void *get(size_t bytes, size_t *cap) {
        size_t c = 64 * 1024;
        while (c < bytes) c <<= 1;
        {
            std::lock_guard<std::mutex> g(mu_);
            auto it = free_.find(c);
            if (it != free_.end()) {
                void *p = it->second;
                free_.erase(it);
                *cap = c;
                return p;
            }
        }
        void *p = nullptr;
        if (cudaMallocHost(&p, c) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        *cap = c;
        return p;
    }
    void put(void *p, size_t cap) {
        if (!p) return;
        std::lock_guard<std::mutex> g(mu_);
        free_.emplace(cap, p);
    }
    ~PinnedPool() {
        for (auto &kv : free_) cudaFreeHost(kv.second);
    }

private:
    std::mutex mu_;
    std::multimap<size_t, void *> free_;
};

// ---------------------------------------------------------------- context engine

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

// ---------------------------------------------------------------- iteration engine

// One unit of an iteration request: a vector (or pair) walking one stream.
struct IterUnit {
    const Rec *stream = nullptr;  // device: first chunk
    int n_chunks = 0;
    int pos = 0;                  // chunks already scheduled
    int8_t kind = SV_VEC;
    int8_t init = INIT_TERMS;     // first slice
    bool rows = false;
    const double *src0 = nullptr, *src1 = nullptr;   // pairs: lambda, rho at the first slice
    double *state = nullptr;
    double *xfree_out = nullptr;
};

struct Req;

struct IterReq {
    Req *r = nullptr;
    int n = 0;
    bool grad = false;
    int phase = 0;                // gradients: 0 = the two half sweeps, 1 = the pair sweeps
    IterUnit u[2];
    int n_units = 0;
    // pinned image (plan, then the result area) and the device block
    unsigned char *h = nullptr;
    size_t h_cap = 0;
    size_t plan_bytes = 0;        // uploaded at admission
    size_t res_off = 0;           // result area in the pinned block
    void *d = nullptr;
    size_t d_bytes = 0;
    // offsets inside the image / device block
    size_t o_recs = 0, o_enc = 0, o_maps = 0, o_midx = 0, o_raw = 0, o_th = 0, o_terms = 0,
           o_pptr = 0, o_prot = 0, o_state = 0, o_grot = 0, o_res = 0;
    int n_enc = 0, n_maps = 0, max_map = 0, n_terms = 0, n_params = 0;
    int64_t s_off[4] = {0, 0, 0, 0};   // record offset of each stream
    int s_chunks[4] = {0, 0, 0, 0};
    int n_streams = 0;
    // device pointers (set at admission)
    const DevTerm *terms = nullptr;
    double *grad_rot = nullptr, *res = nullptr;
    const int32_t *param_ptr = nullptr, *param_rot = nullptr;
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
    IterReq *it = nullptr;
};

}  // namespace

struct stab_server {
    stab_server_opts opts{};
    int device = 0;
    bool iterate = true;
    Hooks hooks;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_queue, cv_done, cv_engine;
    std::deque<Req *> queue;
    std::unordered_map<int64_t, Req *> all;
    std::vector<Req *> active;                // context engine, running
    std::map<int, std::vector<Slot *>> idle;
    std::vector<Slot *> slots;
    std::vector<IterReq *> ready;             // planned, waiting for the engine thread
    int64_t next_id = 0, submitted = 0, completed = 0, bytes_in_use = 0;
    int n_active = 0;
    bool stop = false;
    bool planners_done = false;
    std::vector<std::thread> planners;
    std::thread completer, engine;
    PinnedPool pinned;
};

namespace {

void complete_locked(stab_server *s, Req *r, int status) {
    r->res.status = status;
    r->res.done_s = now_s(s->t0);
    r->done = true;
    s->completed++;
}

void release_locked(stab_server *s, Req *r) {
    if (r->slot) s->idle[r->slot->n].push_back(r->slot);
    r->slot = nullptr;
    if (r->admitted) {
        s->n_active--;
        s->bytes_in_use -= r->footprint;
        r->admitted = false;
    }
}

Slot *make_slot(stab_server *s, int n) {
    Slot *sl = new (std::nothrow) Slot();
    if (!sl) return nullptr;
    stab_opts o;
    stab_default_opts(&o);
    o.device = s->device;
    o.alloc = s->hooks.alloc;
    o.free = s->hooks.free;
    o.alloc_user = s->hooks.user;
    sl->n = n;
    if (stab_create(n, &o, &sl->ctx) != STAB_OK) {
        delete sl;
        return nullptr;
    }
    cudaStream_t st = ctx_stream(sl->ctx);
    sl->d_res = (double *)s->hooks.get(256, st);
    if (!sl->d_res || cudaMallocHost(&sl->h_res, 64 * sizeof(double)) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        if (sl->d_res) s->hooks.put(sl->d_res, 256, st);
        cudaStreamSynchronize(st);
        stab_destroy(sl->ctx);
        if (sl->h_res) cudaFreeHost(sl->h_res);
        delete sl;
        return nullptr;
    }
    return sl;
}

void free_slot(stab_server *s, Slot *sl) {
    if (!sl) return;
    cudaStream_t st = ctx_stream(sl->ctx);
    cudaStreamSynchronize(st);
    s->hooks.put(sl->d_res, 256, st);
    if (sl->d_grads) s->hooks.put(sl->d_grads, sl->grads_cap * 8, st);
    cudaStreamSynchronize(st);
    stab_destroy(sl->ctx);
    if (sl->h_res) cudaFreeHost(sl->h_res);
    if (sl->h_grads) cudaFreeHost(sl->h_grads);
    if (sl->ev) cudaEventDestroy(sl->ev);
    delete sl;
}

// Plans and queues one admitted request on its slot; returns a status.
int launch_on_context(stab_server *s, Req *r) {
    Slot *sl = r->slot;
    const stab_request &q = r->hdr;
    int rc = stab_load_circuit(sl->ctx, q.gates, q.m, q.thetas, q.n_params);
    if (rc == STAB_OK) rc = stab_set_observable(sl->ctx, q.obs, q.n_terms);
    if (rc != STAB_OK) return rc;
    cudaStream_t st = ctx_stream(sl->ctx);
    if (q.kind == STAB_REQ_GRAD) {
        const size_t need = (size_t)(q.n_params > 0 ? q.n_params : 1);
        if (sl->grads_cap < need) {
            // the old buffer may still be read by the slot's last request
            cudaStreamSynchronize(st);
            if (sl->d_grads) s->hooks.put(sl->d_grads, sl->grads_cap * 8, st);
            if (sl->h_grads) cudaFreeHost(sl->h_grads);
            sl->d_grads = nullptr;
            sl->h_grads = nullptr;
            sl->grads_cap = 0;
            sl->d_grads = (double *)s->hooks.get(need * 8, st);
            if (!sl->d_grads) return STAB_E_NOMEM;
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

double aging_bound(const stab_server *s) {
    return s->opts.aging_s == 0.0 ? kDefaultAgingS : s->opts.aging_s;
}

// Position in the queue of the request to admit next (caller holds s->mu).
// The queue is in submission order.  SHORTEST: the least estimated work,
// unless the oldest request has waited longer than the aging bound -- then
// the oldest, so no request waits behind later small ones without limit.
size_t next_request_locked(const stab_server *s) {
    if (s->opts.policy != STAB_SERVE_SHORTEST || s->queue.empty()) return 0;
    const double aging = aging_bound(s);
    if (aging > 0.0 && now_s(s->t0) - s->queue.front()->res.submit_s > aging) return 0;
    size_t best = 0;
    for (size_t i = 1; i < s->queue.size(); ++i)
        if (s->queue[i]->work < s->queue[best]->work) best = i;
    return best;
}

bool use_iteration(const stab_server *s, const Req *r) {
    return s->iterate && r->hdr.n <= s->opts.iter_max_n;
}

// ---------------------------------------------------------------- iteration requests: host side

// Validates and plans a request on the host (planner thread) into a pinned
// image: instruction streams | encoded positions | maps | map gate indices |
// raw gates | angles | terms | slot CSR, then room for the results.
int prepare_iter(stab_server *s, Req *r, IterReq **out) {
    const stab_request &q = r->hdr;
    const int n = q.n;
    int rc = validate_gates(n, q.gates, q.m, q.n_params, nullptr);
    if (rc == STAB_OK) rc = validate_thetas(q.thetas, q.n_params);
    std::vector<DevTerm> terms;
    if (rc == STAB_OK) rc = encode_terms(n, q.obs, q.n_terms, &terms);
    if (rc != STAB_OK) return rc;
    IterReq *it = new (std::nothrow) IterReq();
    if (!it) return STAB_E_NOMEM;
    it->r = r;
    it->n = n;
    it->grad = q.kind == STAB_REQ_GRAD;
    it->n_params = (int)q.n_params;
    HostPlan P;
    std::vector<Rec> S[4];
    std::vector<int32_t> enc[4];
    if (!it->grad) {
        build_plan(n, q.gates, q.m, q.n_params, n <= 4 ? PLAN_ROWS : PLAN_FUSED, &P);
        build_stream(P, true, &S[0], 0, -1, &enc[0]);
        it->n_streams = 1;
    } else {
        // the gradient's split sweeps: rho_0 through [0, cut) and O backward
        // through [cut, P), then the pair backward through [0, cut) and
        // forward through [cut, P)
        build_plan(n, q.gates, q.m, q.n_params, PLAN_GRAD, &P);
        const int np = (int)P.passes.size(), cut = np / 2;
        build_stream(P, false, &S[0], 0, cut, &enc[0]);
        build_stream(P, true, &S[1], cut, np, &enc[1]);
        build_stream(P, true, &S[2], 0, cut, &enc[2]);
        build_stream(P, false, &S[3], cut, np, &enc[3]);
        it->n_streams = 4;
    }
    int64_t n_recs = 0, n_enc = 0;
    for (int k = 0; k < it->n_streams; ++k) {
        it->s_off[k] = n_recs;
        it->s_chunks[k] = (int)(S[k].size() / kChunkRecs);
        n_recs += (int64_t)S[k].size();
        n_enc += (int64_t)enc[k].size();
    }
    if (n_recs > (int64_t)INT32_MAX / 2) {
        delete it;
        return STAB_E_RANGE;
    }
    it->n_enc = (int)n_enc;
    it->n_maps = (int)P.maps.size();
    it->max_map = max_map_count(P.maps.data(), P.maps.size());
    it->n_terms = (int)terms.size();
    size_t o = 0;
    it->o_recs = o;  o += up256((size_t)n_recs * sizeof(Rec));
    it->o_enc = o;   o += up256((size_t)n_enc * 4);
    it->o_maps = o;  o += up256(P.maps.size() * sizeof(DevMap3));
    it->o_midx = o;  o += up256(P.map_gate_idx.size() * 4);
    it->o_raw = o;   o += up256(P.raw.size() * sizeof(RawGate));
    it->o_th = o;    o += up256((size_t)(q.n_params > 0 ? q.n_params : 1) * 8);
    it->o_terms = o; o += up256((terms.size() ? terms.size() : 1) * sizeof(DevTerm));
    it->o_pptr = o;  o += up256(P.param_ptr.size() * 4);
    it->o_prot = o;  o += up256(P.param_rot.size() * 4);
    it->plan_bytes = o;
    const size_t E = (size_t)1 << (2 * n);
    it->o_state = o; o += up256((it->grad ? 12 : 2) * E * 8);
    it->o_grot = o;  o += up256((size_t)(P.n_rot > 0 ? P.n_rot : 1) * 8);
    it->o_res = o;   o += up256((size_t)(1 + (q.n_params > 0 ? q.n_params : 0)) * 8);
    it->d_bytes = o;
    it->res_off = it->plan_bytes;
    const size_t res_bytes = up256((size_t)(1 + (q.n_params > 0 ? q.n_params : 0)) * 8);
    it->h = (unsigned char *)s->pinned.get(it->plan_bytes + res_bytes, &it->h_cap);
    if (!it->h) {
        delete it;
        return STAB_E_NOMEM;
    }
    unsigned char *h = it->h;
    int64_t e = 0;
    for (int k = 0; k < it->n_streams; ++k) {
        std::memcpy(h + it->o_recs + (size_t)it->s_off[k] * sizeof(Rec), S[k].data(),
                    S[k].size() * sizeof(Rec));
        int32_t *ed = (int32_t *)(h + it->o_enc);
        for (int32_t v : enc[k]) ed[e++] = v + (int32_t)it->s_off[k];
    }
    auto put = [&](size_t off, const void *src, size_t bytes) {
        if (bytes) std::memcpy(h + off, src, bytes);
    };
    put(it->o_maps, P.maps.data(), P.maps.size() * sizeof(DevMap3));
    put(it->o_midx, P.map_gate_idx.data(), P.map_gate_idx.size() * 4);
    put(it->o_raw, P.raw.data(), P.raw.size() * sizeof(RawGate));
    put(it->o_th, q.thetas, (size_t)(q.n_params > 0 ? q.n_params : 0) * 8);
    put(it->o_terms, terms.data(), terms.size() * sizeof(DevTerm));
    put(it->o_pptr, P.param_ptr.data(), P.param_ptr.size() * 4);
    put(it->o_prot, P.param_rot.data(), P.param_rot.size() * 4);
    *out = it;
    return STAB_OK;
}

void drop_iter(stab_server *s, IterReq *it) {
    if (!it) return;
    s->pinned.put(it->h, it->h_cap);
    delete it;
}

// ---------------------------------------------------------------- iteration engine thread

struct Flight {
    cudaEvent_t ev = nullptr;
    int slot = 0;
    std::vector<IterReq *> finishing;
    std::vector<int16_t> keys;       // per unit slice: its cost class (see Engine::key)
    std::vector<int32_t> chunks;     // per unit slice: chunks it ran
};

struct Engine {
    stab_server *s = nullptr;
    cudaStream_t st = nullptr;
    int grid_max = 0;
    size_t smem = 0;
    int smem_buf = 0;
    int iter_chunks = kDefaultIterChunks;
    // unit tables, one per slot: pinned copy, device copy, capacity
    ServeUnit *h_tab[kTableSlots] = {};
    ServeUnit *d_tab[kTableSlots] = {};
    int64_t *h_cyc[kTableSlots] = {};      // per unit slice: SM cycles it took (pinned)
    int64_t *d_cyc[kTableSlots] = {};
    int cap[kTableSlots] = {};
    // Adaptive slices: per cost class (n, vector / rows vector / pair, in shared
    // memory or not) an estimate of the SM cycles one chunk takes, learned from
    // the slices' measured lengths; a unit then gets as many chunks as fill the
    // target slice length (0 = no estimate yet: the static budget).
    double est[kCostClasses] = {};
    double target_cycles = 0.0;
    int32_t *d_words = nullptr;         // counters [0, kTableSlots), status at 32
    int32_t *h_status = nullptr;        // pinned, one per slot
    int64_t iterations = 0;
    std::vector<IterReq *> live;
    std::deque<Flight> inflight;
    std::vector<cudaEvent_t> events;

    int init() {
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        int sms = 0, occ = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
        const int kb = s->opts.iter_smem_kb > 0 ? s->opts.iter_smem_kb : kDefaultIterSmemKb;
        smem_buf = kb * 1024;
        smem = serve_smem_bytes(smem_buf);
        if (e == cudaSuccess) e = serve_occupancy(smem, &occ);
        if (e != cudaSuccess || occ < 1) {
            record_cuda_error(e);
            return e == cudaSuccess ? STAB_E_RANGE : STAB_E_CUDA;
        }
        grid_max = sms * std::min(occ, 4);
        if (s->opts.iter_chunks > 0) iter_chunks = s->opts.iter_chunks;
        // the target slice length: iter_slice_us of SM clock (0: the default;
        // < 0: static budgets only)
        int khz = 0;
        if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, s->device) != cudaSuccess) {
            (void)cudaGetLastError();
            khz = 0;
        }
        const double us = s->opts.iter_slice_us == 0.0 ? kDefaultIterSliceUs : s->opts.iter_slice_us;
        target_cycles = (us > 0.0 && khz > 0) ? us * (double)khz / 1000.0 : 0.0;
        d_words = (int32_t *)s->hooks.get(256, st);
        if (!d_words) return STAB_E_NOMEM;
        if (cudaMemsetAsync(d_words, 0, 256, st) != cudaSuccess ||
            cudaMallocHost(&h_status, kTableSlots * sizeof(int32_t)) != cudaSuccess) {
            record_cuda_error(cudaGetLastError());
            return STAB_E_CUDA;
        }
        return STAB_OK;
    }

    void shutdown() {
        if (st) cudaStreamSynchronize(st);
        for (int k = 0; k < kTableSlots; ++k) {
            if (d_tab[k]) s->hooks.put(d_tab[k], (size_t)cap[k] * sizeof(ServeUnit), st);
            if (d_cyc[k]) s->hooks.put(d_cyc[k], (size_t)cap[k] * sizeof(int64_t), st);
            if (h_tab[k]) cudaFreeHost(h_tab[k]);
            if (h_cyc[k]) cudaFreeHost(h_cyc[k]);
        }
        if (d_words) s->hooks.put(d_words, 256, st);
        if (st) cudaStreamSynchronize(st);
        if (h_status) cudaFreeHost(h_status);
        for (cudaEvent_t ev : events) cudaEventDestroy(ev);
        if (st) cudaStreamDestroy(st);
    }

    // Cost class of a unit: n, its kind (vector, rows vector, pair) and whether
    // its vectors fit the launch's shared memory.
    int key(int n, int kind, bool rows) const {
        const size_t E = (size_t)1 << (2 * n);
        const int k = kind != SV_VEC ? 2 : (rows ? 1 : 0);
        const bool smem = (kind != SV_VEC ? 4 : 2) * E * sizeof(double) <= (size_t)smem_buf;
        return (n * 3 + k) * 2 + (smem ? 1 : 0);
    }

    // Chunks a unit runs per iteration.  Static budget: the same work (chunks x
    // 4^n, twice that for a pair) for every unit, iter_chunks chunks at n = 4.
    // Adaptive (a target slice length and an estimate for the unit's class):
    // as many chunks as take about the target length, so the units of one
    // launch end together whatever their size and residency.
    int budget(int n, int kind, bool rows) const {
        const double e = target_cycles > 0.0 ? est[key(n, kind, rows)] : 0.0;
        int64_t c;
        if (e > 0.0) {
            c = (int64_t)(target_cycles / e + 0.5);
        } else {
            c = ((int64_t)iter_chunks << 8) >> (2 * n);
            if (kind != SV_VEC) c /= 2;
        }
        return (int)std::max<int64_t>(1, std::min<int64_t>(c, 4096));
    }

    void finish(IterReq *it, int status) {
        Req *r = it->r;
        if (status == STAB_OK) {
            const double *h = (const double *)(it->h + it->res_off);
            r->res.expect = h[0];
            if (it->grad && it->n_params > 0) r->grads.assign(h + 1, h + 1 + it->n_params);
        }
        if (it->d) s->hooks.put(it->d, it->d_bytes, st);
        drop_iter(s, it);
        r->it = nullptr;
        std::lock_guard<std::mutex> lk(s->mu);
        release_locked(s, r);
        complete_locked(s, r, status);
        s->cv_done.notify_all();
        s->cv_queue.notify_all();
    }

    // Device block, upload and encoding of a newly admitted request; its first units.
    int admit(IterReq *it) {
        it->d = s->hooks.get(it->d_bytes, st);
        if (!it->d) return STAB_E_NOMEM;
        char *d = (char *)it->d;
        cudaError_t e = cudaMemcpyAsync(d, it->h, it->plan_bytes, cudaMemcpyHostToDevice, st);
        Rec *recs = (Rec *)(d + it->o_recs);
        DevMap3 *maps = (DevMap3 *)(d + it->o_maps);
        const double *th = (const double *)(d + it->o_th);
        if (e == cudaSuccess)
            e = launch_compose_maps(maps, it->n_maps, it->max_map, (const int32_t *)(d + it->o_midx),
                                    (const RawGate *)(d + it->o_raw), th, st);
        if (e == cudaSuccess)
            e = launch_encode_stream(recs, (const int32_t *)(d + it->o_enc), it->n_enc, maps, th, st);
        if (e != cudaSuccess) {
            record_cuda_error(e);
            return STAB_E_CUDA;
        }
        it->terms = (const DevTerm *)(d + it->o_terms);
        it->grad_rot = (double *)(d + it->o_grot);
        it->res = (double *)(d + it->o_res);
        it->param_ptr = (const int32_t *)(d + it->o_pptr);
        it->param_rot = (const int32_t *)(d + it->o_prot);
        const size_t E = (size_t)1 << (2 * it->n);
        double *state = (double *)(d + it->o_state);
        if (!it->grad) {
            IterUnit &u = it->u[0];
            u = IterUnit{};
            u.stream = recs + it->s_off[0];
            u.n_chunks = it->s_chunks[0];
            u.kind = SV_VEC;
            u.init = INIT_TERMS;
            u.rows = it->n <= 4;
            u.state = state;
            u.xfree_out = it->res;
            it->n_units = 1;
        } else {
            for (int k = 0; k < 2; ++k) {
                IterUnit &u = it->u[k];
                u = IterUnit{};
                u.stream = recs + it->s_off[k];
                u.n_chunks = it->s_chunks[k];
                u.kind = SV_VEC;
                u.init = k == 0 ? INIT_RHO0 : INIT_TERMS;
                u.state = state + 2 * E * (size_t)k;
            }
            it->n_units = 2;
            it->phase = 0;
        }
        return STAB_OK;
    }

    // The pair sweeps of a gradient, from the vectors its half sweeps left.
    void start_pairs(IterReq *it) {
        const size_t E = (size_t)1 << (2 * it->n);
        double *state = (double *)((char *)it->d + it->o_state);
        const double *rho_mid = state, *lam_mid = state + 2 * E;
        Rec *recs = (Rec *)((char *)it->d + it->o_recs);
        for (int k = 0; k < 2; ++k) {
            IterUnit &u = it->u[k];
            u = IterUnit{};
            u.stream = recs + it->s_off[2 + k];
            u.n_chunks = it->s_chunks[2 + k];
            u.kind = k == 0 ? SV_PAIR_BWD : SV_PAIR_FWD;
            u.init = INIT_LOAD;
            u.src0 = lam_mid;
            u.src1 = rho_mid;
            u.state = state + 4 * E + 4 * E * (size_t)k;
            u.xfree_out = k == 0 ? it->res : nullptr;   // <O>: lambda after the first half
        }
        it->n_units = 2;
        it->phase = 1;
    }

    cudaEvent_t take_event() {
        if (!events.empty()) {
            cudaEvent_t ev = events.back();
            events.pop_back();
            return ev;
        }
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        return ev;
    }

    void retire_front() {
        Flight f = std::move(inflight.front());
        inflight.pop_front();
        cudaError_t e = cudaEventSynchronize(f.ev);
        events.push_back(f.ev);
        int status = STAB_OK;
        if (e != cudaSuccess) {
            record_cuda_error(e);
            status = STAB_E_CUDA;
        } else if (h_status[f.slot] != 0) {
            status = STAB_E_TIMEOUT;
            h_status[f.slot] = 0;
            cudaMemsetAsync(d_words + 32, 0, 4, st);
        } else {
            // what a chunk of each class cost in this launch (running mean
            // weighted toward recent launches)
            for (size_t k = 0; k < f.keys.size(); ++k) {
                const double per = (double)h_cyc[f.slot][k] / (double)std::max(1, f.chunks[k]);
                if (per <= 0.0) continue;
                double &e = est[f.keys[k]];
                e = e > 0.0 ? 0.75 * e + 0.25 * per : per;
            }
        }
        for (IterReq *it : f.finishing) finish(it, status);
    }

    void retire_done() {
        while (!inflight.empty() && cudaEventQuery(inflight.front().ev) == cudaSuccess)
            retire_front();
        (void)cudaGetLastError();
    }

    int ensure_table(int slot, int n_units) {
        if (cap[slot] >= n_units) return STAB_OK;
        int c = std::max(256, cap[slot]);
        while (c < n_units) c *= 2;
        if (d_tab[slot]) s->hooks.put(d_tab[slot], (size_t)cap[slot] * sizeof(ServeUnit), st);
        if (d_cyc[slot]) s->hooks.put(d_cyc[slot], (size_t)cap[slot] * sizeof(int64_t), st);
        if (h_tab[slot]) cudaFreeHost(h_tab[slot]);
        if (h_cyc[slot]) cudaFreeHost(h_cyc[slot]);
        d_tab[slot] = nullptr;
        d_cyc[slot] = nullptr;
        h_tab[slot] = nullptr;
        h_cyc[slot] = nullptr;
        cap[slot] = 0;
        d_tab[slot] = (ServeUnit *)s->hooks.get((size_t)c * sizeof(ServeUnit), st);
        d_cyc[slot] = (int64_t *)s->hooks.get((size_t)c * sizeof(int64_t), st);
        if (!d_tab[slot] || !d_cyc[slot]) return STAB_E_NOMEM;
        if (cudaMallocHost(&h_tab[slot], (size_t)c * sizeof(ServeUnit)) != cudaSuccess ||
            cudaMallocHost(&h_cyc[slot], (size_t)c * sizeof(int64_t)) != cudaSuccess) {
            (void)cudaGetLastError();
            return STAB_E_NOMEM;
        }
        cap[slot] = c;
        return STAB_OK;
    }

    // One launch: a slice of every unit with chunks left.
    int launch_iteration() {
        const int slot = (int)(iterations % kTableSlots);
        struct Item {
            ServeUnit su;
            int64_t cost;
            int16_t key;
        };
        std::vector<Item> items;
        std::vector<IterReq *> finishing, still;
        for (IterReq *it : live) {
            const int E = 1 << (2 * it->n);
            bool left = false;
            for (int k = 0; k < it->n_units; ++k) {
                IterUnit &u = it->u[k];
                if (u.pos >= u.n_chunks) continue;
                const int take = std::min(budget(it->n, u.kind, u.rows), u.n_chunks - u.pos);
                ServeUnit su{};
                su.stream = u.stream + (size_t)u.pos * kChunkRecs;
                su.n_chunks = take;
                su.n = (int8_t)it->n;
                su.kind = u.kind;
                const bool first = u.pos == 0;
                su.init = (int8_t)(first && u.kind == SV_VEC ? u.init : INIT_LOAD);
                su.flags = (int8_t)((u.rows ? SF_ROWS : 0) |
                                    (u.pos + take == u.n_chunks ? SF_LAST : 0));
                su.terms = it->terms;
                su.n_terms = it->n_terms;
                su.src = (first && u.kind != SV_VEC) ? u.src0 : u.state;
                su.src2 = (first && u.kind != SV_VEC) ? u.src1 : u.state + E;
                su.state = u.state;
                su.grad_rot = it->grad_rot;
                su.xfree_out = u.xfree_out;
                // largest slice first: by the class's estimate when there is one
                const int16_t kc = (int16_t)key(it->n, u.kind, u.rows);
                const int64_t cost = est[kc] > 0.0 ? (int64_t)(take * est[kc])
                                                    : (int64_t)take * E * (u.kind == SV_VEC ? 1 : 2);
                items.push_back({su, cost, kc});
                u.pos += take;
                if (u.pos < u.n_chunks) left = true;
            }
            if (left) {
                still.push_back(it);
            } else if (it->grad && it->phase == 0) {
                start_pairs(it);     // scheduled from the next iteration on
                still.push_back(it);
            } else {
                finishing.push_back(it);
            }
        }
        std::stable_sort(items.begin(), items.end(),
                         [](const Item &a, const Item &b) { return a.cost > b.cost; });
        const int n_units = (int)items.size();
        int rc = ensure_table(slot, std::max(n_units, 1));
        if (rc != STAB_OK) return rc;
        for (int k = 0; k < n_units; ++k) h_tab[slot][k] = items[(size_t)k].su;
        cudaError_t e = cudaSuccess;
        if (n_units > 0) {
            e = cudaMemcpyAsync(d_tab[slot], h_tab[slot], (size_t)n_units * sizeof(ServeUnit),
                                cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(d_words + slot, 0, 4, st);
            ServeArgs a{};
            a.units = d_tab[slot];
            a.n_units = n_units;
            a.counter = d_words + slot;
            a.status = d_words + 32;
            a.smem_buf = smem_buf;
            a.unit_cycles = d_cyc[slot];
            if (e == cudaSuccess) e = launch_serve(a, std::min(grid_max, n_units), smem, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_cyc[slot], d_cyc[slot], (size_t)n_units * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, st);
        }
        for (IterReq *it : finishing) {
            if (e != cudaSuccess) break;
            if (it->grad)
                e = launch_gather_grads(it->grad_rot, it->param_ptr, it->param_rot, it->n_params,
                                        it->res + 1, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(it->h + it->res_off, it->res,
                                    (size_t)(1 + (it->grad ? it->n_params : 0)) * 8,
                                    cudaMemcpyDeviceToHost, st);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_status + slot, d_words + 32, 4, cudaMemcpyDeviceToHost, st);
        Flight f;
        f.slot = slot;
        f.ev = e == cudaSuccess ? take_event() : nullptr;
        if (e == cudaSuccess && f.ev) e = cudaEventRecord(f.ev, st);
        if (e != cudaSuccess || !f.ev) {
            record_cuda_error(e);
            cudaStreamSynchronize(st);
            for (IterReq *it : live) finish(it, STAB_E_CUDA);
            live.clear();
            if (f.ev) events.push_back(f.ev);
            return STAB_E_CUDA;
        }
        f.finishing = std::move(finishing);
        f.keys.resize((size_t)n_units);
        f.chunks.resize((size_t)n_units);
        for (int k = 0; k < n_units; ++k) {
            f.keys[(size_t)k] = items[(size_t)k].key;
            f.chunks[(size_t)k] = items[(size_t)k].su.n_chunks;
        }
        inflight.push_back(std::move(f));
        live.swap(still);
        ++iterations;
        return STAB_OK;
    }
};

void engine_main(stab_server *s) {
    cudaSetDevice(s->device);
    Engine E;
    E.s = s;
    const int init_rc = E.init();
    while (true) {
        std::vector<IterReq *> fresh;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (E.live.empty() && E.inflight.empty())
                s->cv_engine.wait(lk, [&] { return !s->ready.empty() || s->planners_done; });
            fresh.swap(s->ready);
            if (fresh.empty() && E.live.empty() && E.inflight.empty() && s->planners_done) break;
        }
        for (IterReq *it : fresh) {
            const int rc = init_rc != STAB_OK ? init_rc : E.admit(it);
            if (rc == STAB_OK) {
                E.live.push_back(it);
            } else {
                if (it->d) cudaStreamSynchronize(E.st);
                E.finish(it, rc);
            }
        }
        E.retire_done();
        if (E.live.empty()) {
            if (!E.inflight.empty()) E.retire_front();
            continue;
        }
        while ((int)E.inflight.size() >= kInFlight) E.retire_front();
        E.launch_iteration();
    }
    E.shutdown();
}

// ---------------------------------------------------------------- planners and completion

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
        if (use_iteration(s, r)) {
            lk.unlock();
            IterReq *it = nullptr;
            const int rc = prepare_iter(s, r, &it);
            lk.lock();
            if (rc != STAB_OK) {
                release_locked(s, r);
                complete_locked(s, r, rc);
                s->cv_done.notify_all();
                s->cv_queue.notify_all();
            } else {
                r->it = it;
                s->ready.push_back(it);
                s->cv_engine.notify_one();
            }
            continue;
        }
        auto &pool = s->idle[r->hdr.n];
        if (!pool.empty()) {
            r->slot = pool.back();
            pool.pop_back();
        }
        lk.unlock();
        int rc = STAB_OK;
        if (!r->slot) {
            r->slot = make_slot(s, r->hdr.n);
            if (!r->slot) rc = STAB_E_NOMEM;
            else {
                std::lock_guard<std::mutex> g(s->mu);
                s->slots.push_back(r->slot);
            }
        }
        if (rc == STAB_OK) rc = launch_on_context(s, r);
        lk.lock();
        if (rc != STAB_OK) {
            if (r->slot) stab_synchronize(r->slot->ctx);
            release_locked(s, r);
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
        if (s->planners_done && s->active.empty()) break;
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
            release_locked(s, r);
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

// n <= 4: the split sweep's transfer matrices (at most two at n = 4, one
// per later part of the chain at n <= 3: bounded by 160 SMs' worth of
// columns), its first-part vectors and the pairs at the cuts.
static int64_t split_sweep_bytes(int n) {
    if (n > 4) return 0;
    const int64_t E = (int64_t)1 << (2 * n);
    int64_t mats = n == 4 ? 2 : std::min<int64_t>(49, 160 / (E - 1));
    if (mats < 1) mats = 1;
    return 8 * (mats * E * E + (n + 1 + 2 * mats) * E);
}

int64_t stab_request_footprint(const stab_request *q) {
    if (!q || q->n < 1 || q->n > STAB_MAX_QUBITS) return 0;
    const int64_t vec = (int64_t)8 << (2 * q->n);
    int64_t fp = (int64_t)q->n * vec;
    // <O>: two vector pairs of the split sweep; gradient: the half-sweep
    // vectors and two (lambda, rho) pairs with their spares (12 vectors)
    const int64_t work = vec * (q->kind == STAB_REQ_GRAD ? 12 : 4);
    if (work > fp) fp = work;
    fp += 96 * (q->m > 0 ? q->m : 0);
    fp += split_sweep_bytes(q->n);
    if (q->kind == STAB_REQ_GRAD && q->n > kMaxResidentAdjoint) {
        // per-CTA partial sums of the streamed adjoint: one per rotation and CTA
        fp += 8 * (q->m > 0 ? q->m : 0) * (int64_t)adjoint_stream_blocks(q->n);
    } else if (q->kind == STAB_REQ_GRAD) {
        // per-thread dot shares of the resident adjoint (at most one rotation
        // per gate), where a context sweep keeps them
        fp += (int64_t)resident_partial_bytes(q->n, q->m > 0 ? q->m : 0);
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
    if ((s->opts.policy != STAB_SERVE_FIFO && s->opts.policy != STAB_SERVE_SHORTEST) ||
        (s->opts.engine != STAB_SERVE_ITERATE && s->opts.engine != STAB_SERVE_CONTEXTS) ||
        s->opts.iter_chunks < 0 || s->opts.iter_smem_kb < 0 || s->opts.iter_smem_kb > 200 ||
        s->opts.iter_max_n < 0 || s->opts.iter_max_n > kServeMaxQubits ||
        !std::isfinite(s->opts.iter_slice_us) || s->opts.iter_slice_us > 1e6 ||
        (s->opts.alloc == nullptr) != (s->opts.free == nullptr)) {
        delete s;
        return STAB_E_INVAL;
    }
    s->iterate = s->opts.engine == STAB_SERVE_ITERATE;
    if (s->opts.iter_max_n == 0) s->opts.iter_max_n = kDefaultIterMaxN;
    s->hooks.alloc = s->opts.alloc;
    s->hooks.free = s->opts.free;
    s->hooks.user = s->opts.alloc_user;
    int dev = s->opts.device;
    cudaError_t e = cudaSuccess;
    if (dev < 0) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        delete s;
        return STAB_E_CUDA;
    }
    s->device = dev;
    s->t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < s->opts.planners; ++i) s->planners.emplace_back(planner_main, s);
    s->completer = std::thread(completer_main, s);
    s->engine = std::thread(engine_main, s);
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

int stab_serve_submit(stab_server *s, const stab_request *req, int64_t *id) {
    return stab_server_submit(s, req, id);
}

int stab_serve_poll(stab_server *s, int64_t id, int32_t *done) {
    return stab_server_poll(s, id, done);
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
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->planners_done = true;
    }
    s->cv_engine.notify_all();
    s->engine.join();
    s->completer.join();
    cudaSetDevice(s->device);
    for (Slot *sl : s->slots) free_slot(s, sl);
    for (auto &kv : s->all) delete kv.second;
    delete s;
    return STAB_OK;
}

}  // extern "C"
