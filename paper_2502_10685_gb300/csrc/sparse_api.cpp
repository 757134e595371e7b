// sparse_api.cpp -- the sparse term-list entry points (include/stab.h): step
// plans, the launch loop with capacity growth, and the switch to the dense
// path once the stabilizer order n' passes a threshold (Sec. II-B, Fig. 1).
//
// A plan is the gate list in application order (backward: reversed, inverse
// gates) cut into steps: maximal runs of Clifford gates (one launch, every
// term mapped in place) and single rotations (four launches, k_sparse.cu).
// The host launches steps ahead without reading the order back: a rotation at
// most doubles n', so from the last order read it knows how many steps cannot
// overflow the buffers or cross the threshold; it then reads the orders and
// the stop flag once.  A step that would overflow is not applied; the buffers
// grow 8x (the list is copied over) and the loop resumes at that step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/stab.h"
#include "launch.h"
#include "planner.h"

using namespace stab;

namespace {

#define SCK(expr)                        \
    do {                                 \
        cudaError_t e_ = (expr);         \
        if (e_ != cudaSuccess) {         \
            record_cuda_error(e_);       \
            return STAB_E_CUDA;          \
        }                                \
    } while (0)

#define SRC(expr)                         \
    do {                                  \
        int r_ = (expr);                  \
        if (r_ != STAB_OK) return r_;     \
    } while (0)

constexpr int64_t kSpMinCap = 4096;
constexpr int64_t kSpMaxCap = 1ll << 30;
constexpr int kSpMinSegment = 16;   // steps launched ahead even when they might stop

struct SpBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

enum { SP_CLIFF = 0, SP_ROT = 1 };

struct SpStep {
    int kind;
    int q, axis, param;       // rotation
    int first, count;         // Clifford run: gates [first, first + count) of the run array
    int tab;                  // Clifford run applied through its tableau (index), or -1
    int64_t gate_lo, gate_hi; // circuit gates [gate_lo, gate_hi) the step covers
};

struct SpPlan {
    std::vector<SpStep> steps;
    std::vector<SpGate> gates;
    std::vector<int32_t> tab_first, tab_count;   // runs that get a tableau
};

// A run of at least this many gates is applied through its tableau (about
// 2n phase products per term) instead of gate by gate.
int tableau_min_gates(int n) { return 2 * n + 8; }

// The outcome of one propagation.
struct SpRun {
    int buf = 0;              // buffer holding the list
    int64_t step = 0;         // the list is the one before this step (== steps: all run)
    int64_t count = 0;
    bool stopped = false;     // threshold reached, or capacity exhausted
};

void build_sp_plan(const std::vector<stab_gate> &gates, bool backward, SpPlan *P) {
    P->steps.clear();
    P->gates.clear();
    const int64_t m = (int64_t)gates.size();
    bool in_run = false;
    for (int64_t k = 0; k < m; ++k) {
        const int64_t i = backward ? m - 1 - k : k;
        const stab_gate &g = gates[i];
        if (g.op >= STAB_RX) {
            SpStep s{};
            s.kind = SP_ROT;
            s.q = g.q0;
            s.axis = g.op - STAB_RX;
            s.param = g.param;
            s.gate_lo = i;
            s.gate_hi = i + 1;
            P->steps.push_back(s);
            in_run = false;
            continue;
        }
        uint8_t op = g.op;
        if (backward && op == STAB_S) op = STAB_SDG;
        else if (backward && op == STAB_SDG) op = STAB_S;
        if (!in_run) {
            SpStep s{};
            s.kind = SP_CLIFF;
            s.first = (int)P->gates.size();
            s.count = 0;
            s.gate_lo = i;
            s.gate_hi = i + 1;
            P->steps.push_back(s);
            in_run = true;
        }
        SpStep &s = P->steps.back();
        P->gates.push_back(SpGate{op, g.q0, g.q1, 0});
        s.count++;
        s.gate_lo = std::min(s.gate_lo, i);
        s.gate_hi = std::max(s.gate_hi, i + 1);
    }
}

void assign_tableaus(int n, SpPlan *P) {
    P->tab_first.clear();
    P->tab_count.clear();
    for (SpStep &s : P->steps) {
        s.tab = -1;
        if (s.kind != SP_CLIFF || s.count < tableau_min_gates(n)) continue;
        s.tab = (int)P->tab_first.size();
        P->tab_first.push_back(s.first);
        P->tab_count.push_back(s.count);
    }
}

}  // namespace

struct stab_sparse {
    int n = 0;
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_st = false;
    stab_opts opts{};
    int64_t max_terms = 0, cap = 0, threshold = 0;
    bool loaded = false;
    std::vector<stab_gate> gates;
    std::vector<double> thetas_h;
    int64_t n_params = 0;
    SpPlan fwd, bwd;
    SpBuf thetas, cs, g_fwd, g_bwd, keys[2], vals[2], table, slot_of, partner, blk, counts,
        flags, partial, scal, dterms, t_fwd, t_bwd, c_fwd, c_bwd, runs;
    int log_h = 0;
    void *pinned = nullptr;
    size_t pinned_bytes = 0;
    std::vector<int64_t> history;
    stab_ctx *dense = nullptr;
    int32_t regrows = 0;
    bool table_dirty = false;   // a run stopped on overflow with slots still claimed

    int dalloc(SpBuf &b, size_t bytes) {
        if (b.p && b.bytes >= bytes) return STAB_OK;
        dfree(b);
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        void *p = nullptr;
        if (opts.alloc) {
            p = opts.alloc(bytes, (void *)st, opts.alloc_user);
            if (!p) return STAB_E_NOMEM;
        } else {
            cudaError_t e = cudaMallocAsync(&p, bytes, st);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                if (e == cudaErrorMemoryAllocation) return STAB_E_NOMEM;
                record_cuda_error(e);
                return STAB_E_CUDA;
            }
        }
        b.p = p;
        b.bytes = bytes;
        return STAB_OK;
    }
    void dfree(SpBuf &b) {
        if (!b.p) return;
        cudaStreamSynchronize(st);
        if (opts.free) opts.free(b.p, b.bytes, (void *)st, opts.alloc_user);
        else cudaFreeAsync(b.p, st);
        b.p = nullptr;
        b.bytes = 0;
    }
    int stage(size_t bytes) {
        if (pinned && pinned_bytes >= bytes) return STAB_OK;
        if (pinned) cudaFreeHost(pinned);
        pinned = nullptr;
        pinned_bytes = 0;
        SCK(cudaMallocHost(&pinned, bytes));
        pinned_bytes = bytes;
        return STAB_OK;
    }

    // Capacity `c` for the list; the live list (count terms in buffer `from`)
    // moves to buffer 0.  The table is twice the capacity, all slots free.
    int reserve(int64_t c, int from, int64_t count) {
        if (c <= cap && from == 0) return STAB_OK;
        c = std::max(c, cap);
        SpBuf nk, nv;
        std::swap(nk, keys[0]);
        std::swap(nv, vals[0]);
        SRC(dalloc(keys[0], (size_t)c * 8));
        SRC(dalloc(vals[0], (size_t)c * 8));
        const SpBuf &ok = from == 0 ? nk : keys[1], &ov = from == 0 ? nv : vals[1];
        if (count > 0) {
            SCK(cudaMemcpyAsync(keys[0].p, ok.p, (size_t)count * 8, cudaMemcpyDeviceToDevice, st));
            SCK(cudaMemcpyAsync(vals[0].p, ov.p, (size_t)count * 8, cudaMemcpyDeviceToDevice, st));
        }
        dfree(nk);
        dfree(nv);
        if (c > cap) {
            SRC(dalloc(keys[1], (size_t)c * 8));
            SRC(dalloc(vals[1], (size_t)c * 8));
            SRC(dalloc(slot_of, (size_t)c * 4));
            SRC(dalloc(partner, (size_t)c * 4));
            int lh = 1;
            while ((1ll << lh) < 2 * c) ++lh;
            SRC(dalloc(table, ((size_t)1 << lh) * sizeof(SpSlot)));
            SCK(cudaMemsetAsync(table.p, 0xff, ((size_t)1 << lh) * sizeof(SpSlot), st));
            log_h = lh;
            cap = c;
        }
        return STAB_OK;
    }

    ~stab_sparse() {
        if (st) cudaStreamSynchronize(st);
        for (SpBuf *b : {&thetas, &cs, &g_fwd, &g_bwd, &keys[0], &keys[1], &vals[0], &vals[1], &table,
                         &slot_of, &partner, &blk, &counts, &flags, &partial, &scal,
                         &dterms, &t_fwd, &t_bwd, &c_fwd, &c_bwd, &runs})
            dfree(*b);
        if (pinned) cudaFreeHost(pinned);
        if (dense) stab_destroy(dense);
        if (own_st && st) cudaStreamDestroy(st);
    }
};

namespace {

// Uploads the initial list to buffer 0 and runs the plan.
int sp_run(stab_sparse *s, const SpPlan &P, const SpBuf &run_gates, const SpBuf &chunks,
           bool backward,
           const std::vector<uint64_t> &k0, const std::vector<double> &v0, SpRun *R,
           int64_t *order_max) {
    const int64_t S = (int64_t)P.steps.size();
    const int64_t n0 = (int64_t)k0.size();
    s->history.clear();
    s->regrows = 0;
    SRC(s->reserve(std::min(s->max_terms, std::max(kSpMinCap, 4 * n0)), 0, 0));
    if (n0 > s->cap) return STAB_E_RANGE;
    if (s->table_dirty) {
        SCK(cudaMemsetAsync(s->table.p, 0xff, ((size_t)1 << s->log_h) * sizeof(SpSlot), s->st));
        s->table_dirty = false;
    }
    SRC(s->dalloc(s->counts, (size_t)(S + 1) * 8));
    SRC(s->stage(std::max<size_t>((size_t)(S + 1) * 8 + 64, (size_t)n0 * 16 + 64)));
    // initial list and order through pinned staging
    char *h = (char *)s->pinned;
    if (n0) {
        std::memcpy(h, k0.data(), (size_t)n0 * 8);
        std::memcpy(h + (size_t)n0 * 8, v0.data(), (size_t)n0 * 8);
        SCK(cudaMemcpyAsync(s->keys[0].p, h, (size_t)n0 * 8, cudaMemcpyHostToDevice, s->st));
        SCK(cudaMemcpyAsync(s->vals[0].p, h + (size_t)n0 * 8, (size_t)n0 * 8,
                            cudaMemcpyHostToDevice, s->st));
    }
    SCK(cudaMemcpyAsync(s->counts.p, &n0, 8, cudaMemcpyHostToDevice, s->st));
    SCK(cudaMemsetAsync(s->flags.p, 0, 16, s->st));
    SCK(cudaStreamSynchronize(s->st));   // the staging buffer is reused below

    std::vector<int> buf_before((size_t)S + 1, 0);
    *order_max = n0;
    int64_t p = 0, known = n0;
    int32_t *flags = (int32_t *)s->flags.p;
    int64_t *counts = (int64_t *)s->counts.p;
    const SpGate *gates = (const SpGate *)run_gates.p;
    while (p < S) {
        const int64_t lim = s->threshold > 0 ? std::min(s->cap, s->threshold) : s->cap;
        // launch steps [p, e): all that cannot pass lim, at least kSpMinSegment
        int64_t e = p, bound = known;
        while (e < S) {
            const SpStep &st = P.steps[e];
            if (st.kind == SP_ROT && 2 * bound > lim && e >= p + kSpMinSegment) break;
            const int cur = buf_before[e];
            if (st.kind == SP_CLIFF && st.tab >= 0) {
                SCK(launch_sp_cliff_tab((uint64_t *)s->keys[cur].p, (double *)s->vals[cur].p,
                                        counts, flags, (int)e, s->n,
                                        (const SpChunk *)chunks.p + (size_t)st.tab * kSpChunkEntries,
                                        bound, s->st));
                buf_before[e + 1] = cur;
            } else if (st.kind == SP_CLIFF) {
                SCK(launch_sp_cliff((uint64_t *)s->keys[cur].p, (double *)s->vals[cur].p,
                                    counts, flags, (int)e, s->n, gates + st.first, st.count,
                                    bound, s->st));
                buf_before[e + 1] = cur;
            } else {
                SpRotArgs a{};
                a.keys = (const uint64_t *)s->keys[cur].p;
                a.vals = (const double *)s->vals[cur].p;
                a.keys_out = (uint64_t *)s->keys[1 - cur].p;
                a.vals_out = (double *)s->vals[1 - cur].p;
                a.counts = counts;
                a.flags = flags;
                a.step = (int32_t)e;
                a.n = s->n;
                a.q = st.q;
                a.axis = st.axis;
                a.cs = (const double *)s->cs.p;
                a.param = st.param;
                a.inverse = backward ? 1 : 0;
                a.table = (SpSlot *)s->table.p;
                a.log_h = s->log_h;
                a.slot_of = (int32_t *)s->slot_of.p;
                a.partner = (int32_t *)s->partner.p;
                a.blk = (int64_t *)s->blk.p;
                a.err = flags + 2;
                a.cap = s->cap;
                a.threshold = s->threshold;
                a.bound = bound;
                SCK(launch_sp_rotation(a, s->st));
                buf_before[e + 1] = 1 - cur;
                bound = std::min(s->cap, 2 * bound);
            }
            ++e;
        }
        // read the orders of steps [p, e] and the flags
        char *hp = (char *)s->pinned;
        SCK(cudaMemcpyAsync(hp, counts + p, (size_t)(e - p + 1) * 8, cudaMemcpyDeviceToHost,
                            s->st));
        SCK(cudaMemcpyAsync(hp + (size_t)(e - p + 1) * 8, flags, 16, cudaMemcpyDeviceToHost,
                            s->st));
        SCK(cudaStreamSynchronize(s->st));
        const int64_t *hc = (const int64_t *)hp;
        const int32_t *hf = (const int32_t *)(hp + (size_t)(e - p + 1) * 8);
        if (hf[2] != 0) return STAB_E_NOMEM;   // a table probe ran out (never expected)
        const int64_t done = hf[0] != 0 ? hf[1] + (hf[0] == 2 ? 1 : 0) : e;
        for (int64_t j = p + 1; j <= done; ++j) {
            s->history.push_back(hc[j - p]);
            *order_max = std::max(*order_max, hc[j - p]);
        }
        if (hf[0] == 1) {
            // step f would overflow: the list before it is intact
            const int64_t f = hf[1];
            const int64_t cnt = hc[f - p];
            if (s->cap >= s->max_terms) {
                s->table_dirty = true;
                R->buf = buf_before[f];
                R->step = f;
                R->count = cnt;
                R->stopped = true;
                return STAB_OK;
            }
            SRC(s->reserve(std::min(s->max_terms, s->cap * 8), buf_before[f], cnt));
            s->regrows++;
            SCK(cudaMemsetAsync(s->flags.p, 0, 16, s->st));
            buf_before[f] = 0;
            p = f;
            known = cnt;
            continue;
        }
        if (hf[0] == 2) {
            const int64_t f = hf[1];
            R->buf = buf_before[f + 1];
            R->step = f + 1;
            R->count = hc[f + 1 - p];
            R->stopped = f + 1 < S;
            return STAB_OK;
        }
        known = hc[e - p];
        p = e;
    }
    R->buf = buf_before[S];
    R->step = S;
    R->count = known;
    R->stopped = false;
    return STAB_OK;
}

int sp_encode_terms(int n, const stab_term *O, int64_t nt, std::vector<uint64_t> *k,
                    std::vector<double> *v) {
    k->clear();
    v->clear();
    if (nt < 0) return STAB_E_RANGE;
    if (nt > 0 && !O) return STAB_E_INVAL;
    const uint64_t lim = n >= 64 ? ~0ull : (1ull << n);
    std::map<uint64_t, double> acc;
    for (int64_t i = 0; i < nt; ++i) {
        if ((n < 64 && (O[i].x >= lim || O[i].z >= lim))) return STAB_E_INVAL;
        if (!std::isfinite(O[i].coeff)) return STAB_E_NONFINITE;
        acc[O[i].z | (O[i].x << n)] += O[i].coeff;
    }
    for (auto &kv : acc) {
        if (kv.second == 0.0) continue;
        k->push_back(kv.first);
        v->push_back(kv.second);
    }
    return STAB_OK;
}

void fill_info(stab_sparse *s, const SpRun &R, int64_t order_max, int64_t dense_gates,
               stab_sparse_info *info) {
    if (!info) return;
    info->order_final = R.count;
    info->order_max = order_max;
    info->steps = (int64_t)s->history.size();
    info->dense_gates = dense_gates;
    info->regrows = s->regrows;
    info->reserved = 0;
}

}  // namespace

extern "C" {

int stab_sparse_create(int n, int64_t max_terms, const stab_opts *opts, stab_sparse **out) {
    if (!out) return STAB_E_INVAL;
    *out = nullptr;
    if (n < 1 || n > STAB_SPARSE_MAX_QUBITS) return STAB_E_RANGE;
    if (max_terms < 1 || max_terms > kSpMaxCap) return STAB_E_RANGE;
    stab_opts o;
    stab_default_opts(&o);
    if (opts) o = *opts;
    if ((o.alloc == nullptr) != (o.free == nullptr)) return STAB_E_INVAL;
    stab_sparse *s = new (std::nothrow) stab_sparse();
    if (!s) return STAB_E_NOMEM;
    s->n = n;
    s->max_terms = max_terms;
    s->threshold = n <= STAB_MAX_QUBITS ? (int64_t)1 << (2 * n - 4 > 0 ? 2 * n - 4 : 0) : 0;
    if (s->threshold >= max_terms) s->threshold = max_terms / 2;
    int dev = o.device;
    cudaError_t e = cudaSuccess;
    if (dev < 0) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e == cudaSuccess) {
        s->device = dev;
        if (o.stream || o.stream_given) {
            s->st = (cudaStream_t)o.stream;
        } else {
            e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
            s->own_st = (e == cudaSuccess);
        }
    }
    if (e != cudaSuccess) {
        record_cuda_error(e);
        delete s;
        return STAB_E_CUDA;
    }
    // the dense context (created on demand) queues on the same stream
    o.device = dev;
    o.stream = (void *)s->st;
    o.stream_given = 1;
    s->opts = o;
    int r = s->dalloc(s->flags, 256);
    if (r == STAB_OK) r = s->dalloc(s->blk, (size_t)kSpMaxBlocks * 8);
    if (r == STAB_OK) r = s->dalloc(s->partial, (size_t)kSpMaxBlocks * 8);
    if (r == STAB_OK) r = s->dalloc(s->scal, 64);
    if (r != STAB_OK) {
        delete s;
        return r;
    }
    *out = s;
    return STAB_OK;
}

int stab_sparse_destroy(stab_sparse *s) {
    if (!s) return STAB_OK;
    cudaSetDevice(s->device);
    delete s;
    return STAB_OK;
}

int stab_sparse_load_circuit(stab_sparse *s, const stab_gate *gates, int64_t m,
                             const double *thetas, int64_t n_params) {
    if (!s) return STAB_E_INVAL;
    SRC(validate_gates(s->n, gates, m, n_params, nullptr));
    SRC(validate_thetas(thetas, n_params));
    SCK(cudaSetDevice(s->device));
    s->loaded = false;
    s->gates.assign(gates, gates + m);
    s->thetas_h.assign(thetas, thetas + n_params);
    s->n_params = n_params;
    build_sp_plan(s->gates, false, &s->fwd);
    build_sp_plan(s->gates, true, &s->bwd);
    assign_tableaus(s->n, &s->fwd);
    assign_tableaus(s->n, &s->bwd);
    const size_t bt = (size_t)std::max<int64_t>(n_params, 1) * 8;
    const size_t bf = std::max<size_t>(s->fwd.gates.size(), 1) * sizeof(SpGate);
    const size_t bb = std::max<size_t>(s->bwd.gates.size(), 1) * sizeof(SpGate);
    const size_t nrf = s->fwd.tab_first.size(), nrb = s->bwd.tab_first.size();
    const size_t br = std::max<size_t>(2 * (nrf + nrb), 1) * 4;
    SRC(s->dalloc(s->thetas, bt));
    SRC(s->dalloc(s->cs, 2 * bt));
    SRC(s->dalloc(s->g_fwd, bf));
    SRC(s->dalloc(s->g_bwd, bb));
    SRC(s->dalloc(s->runs, br));
    SRC(s->dalloc(s->t_fwd, std::max<size_t>(nrf, 1) * 64 * sizeof(SpTab)));
    SRC(s->dalloc(s->t_bwd, std::max<size_t>(nrb, 1) * 64 * sizeof(SpTab)));
    SRC(s->dalloc(s->c_fwd, std::max<size_t>(nrf, 1) * kSpChunkEntries * sizeof(SpChunk)));
    SRC(s->dalloc(s->c_bwd, std::max<size_t>(nrb, 1) * kSpChunkEntries * sizeof(SpChunk)));
    SRC(s->stage(bt + bf + bb + br));
    char *h = (char *)s->pinned;
    std::memcpy(h, s->thetas_h.data(), (size_t)n_params * 8);
    std::memcpy(h + bt, s->fwd.gates.data(), s->fwd.gates.size() * sizeof(SpGate));
    std::memcpy(h + bt + bf, s->bwd.gates.data(), s->bwd.gates.size() * sizeof(SpGate));
    int32_t *hr = (int32_t *)(h + bt + bf + bb);
    std::copy(s->fwd.tab_first.begin(), s->fwd.tab_first.end(), hr);
    std::copy(s->fwd.tab_count.begin(), s->fwd.tab_count.end(), hr + nrf);
    std::copy(s->bwd.tab_first.begin(), s->bwd.tab_first.end(), hr + 2 * nrf);
    std::copy(s->bwd.tab_count.begin(), s->bwd.tab_count.end(), hr + 2 * nrf + nrb);
    SCK(cudaMemcpyAsync(s->thetas.p, h, bt, cudaMemcpyHostToDevice, s->st));
    SCK(launch_sp_cos_sin((const double *)s->thetas.p, n_params, (double *)s->cs.p, s->st));
    SCK(cudaMemcpyAsync(s->g_fwd.p, h + bt, bf, cudaMemcpyHostToDevice, s->st));
    SCK(cudaMemcpyAsync(s->g_bwd.p, h + bt + bf, bb, cudaMemcpyHostToDevice, s->st));
    SCK(cudaMemcpyAsync(s->runs.p, hr, br, cudaMemcpyHostToDevice, s->st));
    const int32_t *dr = (const int32_t *)s->runs.p;
    SCK(launch_sp_tableau((const SpGate *)s->g_fwd.p, dr, dr + nrf, (int)nrf, s->n,
                          (SpTab *)s->t_fwd.p, (SpChunk *)s->c_fwd.p, s->st));
    SCK(launch_sp_tableau((const SpGate *)s->g_bwd.p, dr + 2 * nrf, dr + 2 * nrf + nrb, (int)nrb,
                          s->n, (SpTab *)s->t_bwd.p, (SpChunk *)s->c_bwd.p, s->st));
    SCK(cudaStreamSynchronize(s->st));
    s->loaded = true;
    return STAB_OK;
}

int stab_sparse_set_dense_threshold(stab_sparse *s, int64_t order) {
    if (!s) return STAB_E_INVAL;
    if (order < 0 || (order > 0 && s->n > STAB_MAX_QUBITS)) return STAB_E_RANGE;
    s->threshold = order;
    return STAB_OK;
}

int stab_sparse_expect(stab_sparse *s, const stab_term *O, int64_t n_terms, double *out,
                       stab_sparse_info *info) {
    if (!s || !out) return STAB_E_INVAL;
    if (!s->loaded) return STAB_E_STATE;
    SCK(cudaSetDevice(s->device));
    std::vector<uint64_t> k0;
    std::vector<double> v0;
    SRC(sp_encode_terms(s->n, O, n_terms, &k0, &v0));
    SpRun R;
    int64_t order_max = 0;
    if (k0.empty()) {
        s->history.clear();
        *out = 0.0;
        fill_info(s, R, 0, -1, info);
        return STAB_OK;
    }
    SRC(sp_run(s, s->bwd, s->g_bwd, s->c_bwd, true, k0, v0, &R, &order_max));
    int64_t dense_gates = -1;
    if (R.stopped) {
        // the rest of the circuit (backward: gates [0, g)) on the dense vector
        if (s->n > STAB_MAX_QUBITS) return STAB_E_RANGE;
        const int64_t g = s->bwd.steps[R.step].gate_hi;
        if (!s->dense) SRC(stab_create(s->n, &s->opts, &s->dense));
        SRC(stab_load_circuit(s->dense, s->gates.data(), g, s->thetas_h.data(), s->n_params));
        SRC(s->dalloc(s->dterms, (size_t)std::max<int64_t>(R.count, 1) * sizeof(DevTerm)));
        SCK(launch_sp_to_terms((const uint64_t *)s->keys[R.buf].p,
                               (const double *)s->vals[R.buf].p, (const int64_t *)s->counts.p,
                               (int)R.step, (DevTerm *)s->dterms.p, R.count, s->st));
        SRC(expect_device_terms(s->dense, (const DevTerm *)s->dterms.p, R.count, out));
        dense_gates = g;
    } else {
        SCK(launch_sp_xfree((const uint64_t *)s->keys[R.buf].p, (const double *)s->vals[R.buf].p,
                            (const int64_t *)s->counts.p, (int)R.step, s->n,
                            (double *)s->partial.p, (double *)s->scal.p, s->st));
        SCK(cudaMemcpyAsync(s->pinned, s->scal.p, 8, cudaMemcpyDeviceToHost, s->st));
        SCK(cudaStreamSynchronize(s->st));
        std::memcpy(out, s->pinned, 8);
    }
    fill_info(s, R, order_max, dense_gates, info);
    return STAB_OK;
}

int stab_sparse_generator(stab_sparse *s, int k, int64_t max_out, stab_term *out,
                          int64_t *n_out, stab_sparse_info *info) {
    if (!s || !n_out || max_out < 0 || (max_out > 0 && !out)) return STAB_E_INVAL;
    if (!s->loaded) return STAB_E_STATE;
    if (k < 0 || k >= s->n) return STAB_E_RANGE;
    SCK(cudaSetDevice(s->device));
    const std::vector<uint64_t> k0 = {1ull << k};
    const std::vector<double> v0 = {1.0};
    const int64_t keep = s->threshold;
    s->threshold = 0;   // generators stay on the list
    SpRun R;
    int64_t order_max = 0;
    const int r = sp_run(s, s->fwd, s->g_fwd, s->c_fwd, false, k0, v0, &R, &order_max);
    s->threshold = keep;
    SRC(r);
    if (R.stopped) return STAB_E_RANGE;
    *n_out = R.count;
    fill_info(s, R, order_max, -1, info);
    if (R.count > max_out) return STAB_E_RANGE;
    if (R.count == 0) return STAB_OK;
    SRC(s->stage((size_t)R.count * 16));
    char *h = (char *)s->pinned;
    SCK(cudaMemcpyAsync(h, s->keys[R.buf].p, (size_t)R.count * 8, cudaMemcpyDeviceToHost, s->st));
    SCK(cudaMemcpyAsync(h + (size_t)R.count * 8, s->vals[R.buf].p, (size_t)R.count * 8,
                        cudaMemcpyDeviceToHost, s->st));
    SCK(cudaStreamSynchronize(s->st));
    const uint64_t *hk = (const uint64_t *)h;
    const double *hv = (const double *)(h + (size_t)R.count * 8);
    const uint64_t zmask = (s->n >= 64) ? ~0ull : ((1ull << s->n) - 1);
    for (int64_t i = 0; i < R.count; ++i) {
        out[i].coeff = hv[i];
        out[i].x = hk[i] >> s->n;
        out[i].z = hk[i] & zmask;
    }
    return STAB_OK;
}

int stab_sparse_order_history(stab_sparse *s, int64_t *orders, int64_t max, int64_t *count) {
    if (!s || !count || max < 0 || (max > 0 && !orders)) return STAB_E_INVAL;
    const int64_t c = (int64_t)s->history.size();
    *count = c;
    for (int64_t i = 0; i < std::min(c, max); ++i) orders[i] = s->history[(size_t)i];
    return STAB_OK;
}

}  // extern "C"
