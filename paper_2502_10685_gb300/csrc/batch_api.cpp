// batch_api.cpp -- stab_batch_*: many uneven circuits in one persistent launch.
//
// Create plans every item, concatenates all instruction streams, angle
// arrays, map gate lists and observable terms into one device buffer (one
// host-to-device copy), encodes every rotation and map with one launch, and
// builds the unit table (one unit per propagated vector) sorted longest
// first.  Run replays a CUDA graph holding the counter reset and the
// persistent launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "../../include/stab.h"
#include "host_pool.h"
#include "launch.h"
#include "planner.h"

using namespace stab;

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

struct stab_batch {
    int device = 0;
    cudaStream_t st = nullptr;        // internal stream: capture and launches
    cudaStream_t user_st = nullptr;   // caller's stream, joined by events
    bool has_user_st = false;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    bool own_st = false;
    stab_alloc_fn alloc = nullptr;
    stab_free_fn free = nullptr;
    void *user = nullptr;

    int64_t count = 0;
    std::vector<int32_t> item_n, item_kind;
    std::vector<int64_t> gen_off;     // doubles into the generator buffer (-1: none)
    int n_units = 0;
    int max_n = 1;
    int grid = 0;
    int ctas_per_sm = 1;
    int smem_n = kMaxResidentQubits;   // vectors up to this n in shared memory, larger in the slab
    size_t smem = 0;

    Buf data, gens, exps, slab, counter;   // counter also holds the status word
    const BatchUnit *units_dev = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool ran = false;

    int dalloc(Buf &b, size_t bytes) {
        bytes = up256(bytes ? bytes : 256);
        void *p = nullptr;
        if (alloc) {
            p = alloc(bytes, (void *)st, user);
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
    void dfree(Buf &b) {
        if (!b.p) return;
        if (free) free(b.p, b.bytes, (void *)st, user);
        else cudaFreeAsync(b.p, st);
        b.p = nullptr;
        b.bytes = 0;
    }
};

namespace {

#define BCK(expr)                       \
    do {                                \
        cudaError_t e_ = (expr);        \
        if (e_ != cudaSuccess) {        \
            record_cuda_error(e_);      \
            return STAB_E_CUDA;         \
        }                               \
    } while (0)

#define BRC(expr)                        \
    do {                                 \
        int r_ = (expr);                 \
        if (r_ != STAB_OK) return r_;    \
    } while (0)

int launch_graph_or_direct(stab_batch *b, const BatchArgs &a, int grid, bool use_graph) {
    if (!use_graph) {
        BCK(cudaMemsetAsync(a.counter, 0, sizeof(int32_t), b->st));
        BCK(launch_batch(a, grid, b->smem, b->st));
        return STAB_OK;
    }
    if (!b->graph) {
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = cudaMemsetAsync(a.counter, 0, sizeof(int32_t), b->st);
        cudaError_t e2 = e1 == cudaSuccess ? launch_batch(a, grid, b->smem, b->st) : e1;
        cudaError_t e3 = cudaStreamEndCapture(b->st, &g);
        if (e2 != cudaSuccess || e3 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            record_cuda_error(e2 != cudaSuccess ? e2 : e3);
            return STAB_E_CUDA;
        }
        cudaError_t e4 = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        BCK(e4);
    }
    BCK(cudaGraphLaunch(b->graph, b->st));
    return STAB_OK;
}

BatchArgs make_args(stab_batch *b, int n_units) {
    BatchArgs a{};
    a.units = b->units_dev;
    a.n_units = n_units;
    a.counter = (int32_t *)b->counter.p;
    a.status = (int32_t *)b->counter.p + 32;
    a.slab = (double *)b->slab.p;
    a.slab_doubles = b->max_n > b->smem_n ? (size_t)2 << (2 * b->max_n) : 0;
    a.smem_n = b->smem_n;
    return a;
}

// Picks the residency -- which vectors live in shared memory (n <= smem_n)
// rather than in the CTA's slab, and how many CTAs run per SM -- by timing the
// persistent launch on a prefix of the unit table (the longest units, one per
// CTA of the widest candidate) for every candidate pair; one untimed launch
// first.  Each sampled unit runs only its first kTuneChunks chunks: the choice
// rests on the per-pass rate of each residency, and whole streams of the
// longest circuits made the tuning cost seconds.  (The partial outputs are
// overwritten by the first real run.)
constexpr int kTuneChunks = 24;

struct Residency {
    int smem_n;
    size_t smem;
    int max_occ;
};

int autotune(stab_batch *b, int sms, const std::vector<Residency> &res) {
    int widest = 1;
    for (const Residency &r : res) widest = std::max(widest, r.max_occ);
    const int sample = std::min(b->n_units, sms * widest);
    float best = 1e30f;
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    bool warm = false;
    Residency tuned = res[0];
    for (const Residency &r : res) {
        std::vector<int> cands;
        for (int occ : {1, 2, 4, r.max_occ})
            if (occ <= r.max_occ && std::find(cands.begin(), cands.end(), occ) == cands.end())
                cands.push_back(occ);
        b->smem_n = r.smem_n;
        b->smem = r.smem;
        for (int occ : cands) {
            BatchArgs a = make_args(b, sample);
            a.max_chunks = kTuneChunks;
            if (!warm) {
                BRC(launch_graph_or_direct(b, a, sms * occ, false));
                warm = true;
            }
            BCK(cudaEventRecord(e0, b->st));
            BRC(launch_graph_or_direct(b, a, sms * occ, false));
            BCK(cudaEventRecord(e1, b->st));
            BCK(cudaEventSynchronize(e1));
            float ms = 0;
            BCK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                b->ctas_per_sm = occ;
                tuned = r;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->smem_n = tuned.smem_n;
    b->smem = tuned.smem;
    return STAB_OK;
}

int build(stab_batch *b, const stab_batch_item *items, int64_t count, int kernel) {
    std::vector<Rec> recs;
    std::vector<int32_t> enc;
    std::vector<DevMap3> maps;
    std::vector<int32_t> midx;
    std::vector<RawGate> raw;
    std::vector<double> thetas;
    std::vector<DevTerm> terms;
    struct UnitPlan {
        int64_t rec_off, n_chunks, term_off, n_terms, item;
        int n, init, gen;
        int64_t cost;
    };
    std::vector<UnitPlan> ups;
    b->item_n.resize(count);
    b->item_kind.resize(count);
    b->gen_off.assign(count, -1);
    int64_t gens_doubles = 0;
    for (int64_t it = 0; it < count; ++it) {
        const stab_batch_item &I = items[it];
        if (I.n < 1 || I.n > STAB_BATCH_MAX_QUBITS) return STAB_E_RANGE;
        if (I.kind != STAB_ITEM_GENERATORS && I.kind != STAB_ITEM_EXPECT) return STAB_E_INVAL;
    }
    // Plans and instruction streams of the items, built on host threads (each
    // item is independent); then concatenated in item order below.
    struct ItemPlan {
        HostPlan P;
        std::vector<Rec> S;
        std::vector<DevTerm> t;
        int64_t n_enc = 0;           // R_ROT and R_MAP3 records of S (filled by the encoder)
        int rc = STAB_OK;
    };
    std::vector<ItemPlan> plans((size_t)count);
    {
        std::atomic<int64_t> next{0};
        auto worker = [&]() {
            std::vector<int32_t> enc_pos;   // positions of the encoded records (counted only)
            for (int64_t it = next++; it < count; it = next++) {
                const stab_batch_item &I = items[it];
                ItemPlan &ip = plans[(size_t)it];
                ip.rc = validate_gates(I.n, I.gates, I.m, I.n_params, nullptr);
                if (ip.rc == STAB_OK) ip.rc = validate_thetas(I.thetas, I.n_params);
                if (ip.rc == STAB_OK && I.kind == STAB_ITEM_EXPECT)
                    ip.rc = encode_terms(I.n, I.obs, I.n_terms, &ip.t);
                if (ip.rc != STAB_OK) continue;
                build_plan(I.n, I.gates, I.m, I.n_params, I.n <= 4 ? PLAN_ROWS : PLAN_FUSED,
                           &ip.P);
                build_stream(ip.P, I.kind == STAB_ITEM_EXPECT, &ip.S, 0, -1, &enc_pos);
                ip.n_enc = (int64_t)enc_pos.size();
            }
        };
        const unsigned hw = std::thread::hardware_concurrency();
        const int n_threads = (int)std::max(1u, std::min(hw ? hw : 1u, 16u));
        std::vector<std::thread> pool;
        for (int k = 1; k < n_threads && k < count; ++k) pool.emplace_back(worker);
        worker();
        for (auto &t : pool) t.join();
    }
    for (int64_t it = 0; it < count; ++it) BRC(plans[(size_t)it].rc);
    // Concatenation in item order: offsets first, then every item's records,
    // maps and gate indices copied (references offset) on the host pool.
    struct Off {
        int64_t rec, enc, map, midx, raw, th, term;
    };
    std::vector<Off> off((size_t)count);
    Off tot{0, 0, 0, 0, 0, 0, 0};
    for (int64_t it = 0; it < count; ++it) {
        const ItemPlan &ip = plans[(size_t)it];
        off[(size_t)it] = tot;
        tot.rec += (int64_t)ip.S.size();
        tot.enc += ip.n_enc;
        tot.map += (int64_t)ip.P.maps.size();
        tot.midx += (int64_t)ip.P.map_gate_idx.size();
        tot.raw += (int64_t)ip.P.raw.size();
        tot.th += items[it].n_params;
        tot.term += (int64_t)ip.t.size();
    }
    if (tot.rec > (int64_t)INT32_MAX / 2) return STAB_E_RANGE;
    recs.resize((size_t)tot.rec);
    enc.resize((size_t)tot.enc);
    maps.resize((size_t)tot.map);
    midx.resize((size_t)tot.midx);
    raw.resize((size_t)tot.raw);
    thetas.resize((size_t)tot.th);
    terms.resize((size_t)tot.term);
    {
        std::vector<std::function<void()>> jobs;
        const int64_t per = std::max<int64_t>(1, count / 64);
        for (int64_t lo = 0; lo < count; lo += per) {
            const int64_t hi = std::min(count, lo + per);
            jobs.push_back([&, lo, hi] {
                for (int64_t it = lo; it < hi; ++it) {
                    const stab_batch_item &I = items[it];
                    const ItemPlan &ip = plans[(size_t)it];
                    const Off &o = off[(size_t)it];
                    const std::vector<Rec> &S = ip.S;
                    int64_t e = o.enc;
                    for (size_t i = 0; i < S.size(); ++i) {
                        Rec r = S[i];
                        if (r.kind == R_ROT) {
                            r.param += (int32_t)o.th;
                            enc[(size_t)e++] = (int32_t)(o.rec + (int64_t)i);
                        } else if (r.kind == R_MAP3) {
                            r.param += (int32_t)o.map;
                            enc[(size_t)e++] = (int32_t)(o.rec + (int64_t)i);
                        }
                        recs[(size_t)o.rec + i] = r;
                    }
                    for (size_t i = 0; i < ip.P.maps.size(); ++i) {
                        DevMap3 mp = ip.P.maps[i];
                        mp.first += (int32_t)o.midx;
                        maps[(size_t)o.map + i] = mp;
                    }
                    for (size_t i = 0; i < ip.P.map_gate_idx.size(); ++i)
                        midx[(size_t)o.midx + i] = ip.P.map_gate_idx[i] + (int32_t)o.raw;
                    for (size_t i = 0; i < ip.P.raw.size(); ++i) {
                        RawGate g = ip.P.raw[i];
                        if (g.op >= STAB_RX) g.param += (int32_t)o.th;
                        raw[(size_t)o.raw + i] = g;
                    }
                    std::copy(I.thetas, I.thetas + I.n_params, thetas.begin() + (ptrdiff_t)o.th);
                    std::copy(ip.t.begin(), ip.t.end(), terms.begin() + (ptrdiff_t)o.term);
                }
            });
        }
        HostPool::run(jobs);
    }
    for (int64_t it = 0; it < count; ++it) {
        const stab_batch_item &I = items[it];
        b->item_n[it] = I.n;
        b->item_kind[it] = I.kind;
        b->max_n = std::max(b->max_n, (int)I.n);
        const ItemPlan &ip = plans[(size_t)it];
        const Off &o = off[(size_t)it];
        const int64_t n_chunks = (int64_t)ip.S.size() / kChunkRecs;
        const int64_t cost = n_chunks * ((int64_t)1 << (2 * I.n));
        if (I.kind == STAB_ITEM_GENERATORS) {
            b->gen_off[it] = gens_doubles;
            for (int k = 0; k < I.n; ++k)
                ups.push_back({o.rec, n_chunks, 0, 0, it, I.n, INIT_GENERATOR, k, cost});
            gens_doubles += (int64_t)I.n << (2 * I.n);
        } else {
            ups.push_back({o.rec, n_chunks, o.term, (int64_t)ip.t.size(), it, I.n, INIT_TERMS, 0,
                           cost});
        }
    }
    plans.clear();   // the items' host plans
    plans.shrink_to_fit();
    std::stable_sort(ups.begin(), ups.end(),
                     [](const UnitPlan &x, const UnitPlan &y) { return x.cost > y.cost; });
    b->n_units = (int)ups.size();

    // one device buffer: recs | enc | maps | midx | raw | thetas | terms | units
    const size_t o_recs = 0;
    const size_t o_enc = o_recs + up256(recs.size() * sizeof(Rec));
    const size_t o_maps = o_enc + up256(enc.size() * 4);
    const size_t o_midx = o_maps + up256(maps.size() * sizeof(DevMap3));
    const size_t o_raw = o_midx + up256(midx.size() * 4);
    const size_t o_th = o_raw + up256(raw.size() * sizeof(RawGate));
    const size_t o_terms = o_th + up256(thetas.size() * 8);
    const size_t o_units = o_terms + up256(terms.size() * sizeof(DevTerm));
    const size_t total = o_units + up256(ups.size() * sizeof(BatchUnit));
    BRC(b->dalloc(b->data, total));
    BRC(b->dalloc(b->gens, (size_t)std::max<int64_t>(gens_doubles, 1) * 8));
    BRC(b->dalloc(b->exps, (size_t)count * 8));
    BRC(b->dalloc(b->counter, 256));
    BCK(cudaMemsetAsync(b->counter.p, 0, 256, b->st));
    char *d = (char *)b->data.p;
    std::vector<BatchUnit> units(ups.size());
    for (size_t k = 0; k < ups.size(); ++k) {
        const UnitPlan &u = ups[k];
        BatchUnit U{};
        U.stream = (const Rec *)(d + o_recs) + u.rec_off;
        U.n_chunks = (int32_t)u.n_chunks;
        U.n = (int8_t)u.n;
        U.init = (int8_t)u.init;
        U.gen = (int16_t)u.gen;
        U.terms = (const DevTerm *)(d + o_terms) + u.term_off;
        U.n_terms = (int32_t)u.n_terms;
        if (u.init == INIT_GENERATOR) {
            U.out = (double *)b->gens.p + b->gen_off[u.item] + ((int64_t)u.gen << (2 * u.n));
        } else {
            U.xfree_out = (double *)b->exps.p + u.item;
        }
        U.cost = u.cost;
        units[k] = U;
    }
    void *h = nullptr;
    BCK(cudaMallocHost(&h, total));
    char *hc = (char *)h;
    auto put = [&](size_t off, const void *src, size_t bytes) {
        if (bytes) std::memcpy(hc + off, src, bytes);
    };
    put(o_recs, recs.data(), recs.size() * sizeof(Rec));
    put(o_enc, enc.data(), enc.size() * 4);
    put(o_maps, maps.data(), maps.size() * sizeof(DevMap3));
    put(o_midx, midx.data(), midx.size() * 4);
    put(o_raw, raw.data(), raw.size() * sizeof(RawGate));
    put(o_th, thetas.data(), thetas.size() * 8);
    put(o_terms, terms.data(), terms.size() * sizeof(DevTerm));
    put(o_units, units.data(), units.size() * sizeof(BatchUnit));
    cudaError_t e = cudaMemcpyAsync(d, h, total, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
        e = launch_compose_maps((DevMap3 *)(d + o_maps), (int)maps.size(),
                                max_map_count(maps.data(), maps.size()),
                                (const int32_t *)(d + o_midx), (const RawGate *)(d + o_raw),
                                (const double *)(d + o_th), b->st);
    if (e == cudaSuccess && !enc.empty())
        e = launch_encode_stream((Rec *)(d + o_recs), (const int32_t *)(d + o_enc), (int)enc.size(),
                                 (const DevMap3 *)(d + o_maps), (const double *)(d + o_th), b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    cudaFreeHost(h);
    BCK(e);
    b->units_dev = (const BatchUnit *)(d + o_units);

    // residency: shared memory for the vectors of n <= smem_n, a global slab
    // per CTA above.  Candidates: smem_n = min(max n, 6) and, with AUTO, also
    // 5 and 4 (less shared memory per CTA, so more CTAs per SM, at the cost of
    // n = 5, 6 vectors in L2-resident slabs); the autotuner times them.
    // RESIDENT keeps min(max n, 6); STREAMED takes 4 (every n >= 5 vector in a slab).
    int sms = 0;
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    std::vector<Residency> res;
    const int top = std::min(b->max_n, kMaxResidentQubits);
    const int lo = kernel == STAB_KERNEL_AUTO ? std::max(4, top - 2)
                   : kernel == STAB_KERNEL_STREAMED ? std::min(4, top) : top;
    const int hi = kernel == STAB_KERNEL_STREAMED ? std::min(4, top) : top;
    for (int sn = hi; sn >= lo; --sn) {
        Residency r{sn, batch_smem_bytes(sn), 1};
        BCK(batch_occupancy(r.smem, &r.max_occ));
        if (r.max_occ < 1) continue;
        r.max_occ = std::min(r.max_occ, 8);
        res.push_back(r);
    }
    if (res.empty()) return STAB_E_RANGE;
    // the slabs of all resident CTAs of the widest candidate that needs them
    int slab_ctas = 0;
    for (const Residency &r : res)
        if (b->max_n > r.smem_n) slab_ctas = std::max(slab_ctas, sms * r.max_occ);
    if (slab_ctas > 0) {
        const size_t per = (size_t)2 << (2 * b->max_n);
        BRC(b->dalloc(b->slab, per * 8 * (size_t)slab_ctas));
    }
    b->smem_n = res[0].smem_n;
    b->smem = res[0].smem;
    b->ctas_per_sm = res[0].max_occ;
    if (kernel == STAB_KERNEL_AUTO && (res.size() > 1 || res[0].max_occ > 1))
        BRC(autotune(b, sms, res));
    b->grid = sms * b->ctas_per_sm;
    return STAB_OK;
}

}  // namespace

extern "C" {

int stab_batch_create(const stab_batch_item *items, int64_t count, const stab_opts *opts,
                      stab_batch **out) {
    if (!out) return STAB_E_INVAL;
    *out = nullptr;
    if (count < 1 || count > (int64_t)INT32_MAX / 16) return STAB_E_RANGE;
    if (!items) return STAB_E_INVAL;
    stab_opts o;
    stab_default_opts(&o);
    if (opts) o = *opts;
    if ((o.alloc == nullptr) != (o.free == nullptr)) return STAB_E_INVAL;
    stab_batch *b = new (std::nothrow) stab_batch();
    if (!b) return STAB_E_NOMEM;
    b->alloc = o.alloc;
    b->free = o.free;
    b->user = o.alloc_user;
    b->count = count;
    int dev = o.device;
    cudaError_t e = cudaSuccess;
    if (dev < 0) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e == cudaSuccess) {
        b->device = dev;
        // the persistent launch is captured into a graph, which the legacy
        // default stream cannot do: run on an own stream and join the
        // caller's stream with events
        b->has_user_st = o.stream != nullptr || o.stream_given;
        b->user_st = (cudaStream_t)o.stream;
        e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
        b->own_st = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        stab_batch_destroy(b);
        return STAB_E_CUDA;
    }
    const int rc = build(b, items, count, o.kernel);
    if (rc != STAB_OK) {
        stab_batch_destroy(b);
        return rc;
    }
    *out = b;
    return STAB_OK;
}

int stab_batch_run(stab_batch *b) {
    if (!b) return STAB_E_INVAL;
    BCK(cudaSetDevice(b->device));
    const BatchArgs a = make_args(b, b->n_units);
    if (b->has_user_st) {
        BCK(cudaEventRecord(b->ev_in, b->user_st));
        BCK(cudaStreamWaitEvent(b->st, b->ev_in, 0));
    }
    BRC(launch_graph_or_direct(b, a, b->grid, true));
    if (b->has_user_st) {
        BCK(cudaEventRecord(b->ev_out, b->st));
        BCK(cudaStreamWaitEvent(b->user_st, b->ev_out, 0));
    }
    b->ran = true;
    return STAB_OK;
}

int stab_apply_batch(stab_batch *b) { return stab_batch_run(b); }

static int batch_status(stab_batch *b) {
    int32_t h = 0;
    BCK(cudaMemcpyAsync(&h, (int32_t *)b->counter.p + 32, 4, cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    if (h != 0) {
        BCK(cudaMemsetAsync((int32_t *)b->counter.p + 32, 0, 4, b->st));
        return STAB_E_TIMEOUT;
    }
    return STAB_OK;
}

int stab_batch_expectations(stab_batch *b, double *out) {
    if (!b || !out) return STAB_E_INVAL;
    if (!b->ran) return STAB_E_STATE;
    BCK(cudaSetDevice(b->device));
    std::vector<double> h((size_t)b->count);
    BCK(cudaMemcpyAsync(h.data(), b->exps.p, (size_t)b->count * 8, cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    BRC(batch_status(b));
    for (int64_t i = 0; i < b->count; ++i)
        out[i] = b->item_kind[i] == STAB_ITEM_EXPECT ? h[i] : std::nan("");
    return STAB_OK;
}

int stab_batch_generators(stab_batch *b, int64_t item, double *out, int out_is_device) {
    if (!b || !out || item < 0 || item >= b->count) return STAB_E_INVAL;
    if (b->gen_off[item] < 0) return STAB_E_INVAL;
    if (!b->ran) return STAB_E_STATE;
    BCK(cudaSetDevice(b->device));
    const int n = b->item_n[item];
    const size_t bytes = ((size_t)n << (2 * n)) * 8;
    const double *src = (const double *)b->gens.p + b->gen_off[item];
    if (out_is_device) {
        BCK(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToDevice, b->st));
        return STAB_OK;
    }
    BCK(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    return batch_status(b);
}

int stab_batch_info(stab_batch *b, int64_t *units, int32_t *grid, int32_t *ctas_per_sm,
                    int32_t *smem_max_n) {
    if (!b) return STAB_E_INVAL;
    if (units) *units = b->n_units;
    if (grid) *grid = b->grid;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    if (smem_max_n) *smem_max_n = b->smem_n;
    return STAB_OK;
}

int stab_batch_destroy(stab_batch *b) {
    if (!b) return STAB_OK;
    cudaSetDevice(b->device);
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->dfree(b->data);
    b->dfree(b->gens);
    b->dfree(b->exps);
    b->dfree(b->slab);
    b->dfree(b->counter);
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->own_st && b->st) cudaStreamDestroy(b->st);
    delete b;
    return STAB_OK;
}

}  // extern "C"
