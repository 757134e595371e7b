// stab_api.cpp -- the C interface (include/stab.h): contexts, device buffers,
// circuit loading, and the launch sequences of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/stab.h"
#include "launch.h"
#include "host_pool.h"
#include "planner.h"
#include "tuner.h"

using namespace stab;

namespace {

thread_local int g_last_cuda = 0;

}  // namespace

void stab::record_cuda_error(cudaError_t e) { g_last_cuda = (int)e; }

namespace {

#define CK(expr)                                                    \
    do {                                                            \
        cudaError_t e_ = (expr);                                    \
        if (e_ != cudaSuccess) {                                    \
            g_last_cuda = (int)e_;                                  \
            return STAB_E_CUDA;                                     \
        }                                                           \
    } while (0)

#define RC(expr)                 \
    do {                         \
        int r_ = (expr);         \
        if (r_ != STAB_OK) return r_; \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Resident plans with at least this many passes also get split streams.
constexpr int kSplitMinPasses = 64;
// Resident adjoint: per-thread dot shares while the CTA has at most this many
// threads (n <= 5) and the shares take at most this many bytes.
constexpr int kPartialThreads = 256;
constexpr size_t kPartialBytes = (size_t)256 << 20;

}  // namespace

size_t stab::resident_partial_bytes(int n, int64_t n_rot) {
    const int t = resident_adjoint_threads(n);
    const size_t rows = (size_t)(n_rot > 0 ? n_rot : 0), cols = (size_t)(t > 0 ? t : 0);
    const size_t bytes = rows * cols * sizeof(double);
    return (t > 0 && t <= kPartialThreads && bytes <= kPartialBytes) ? bytes : 0;
}

namespace {

// Plans of at least this many passes build their instruction streams on
// several host threads.
constexpr int kThreadedStreamPasses = 2048;

// Instruction stream of a plan for the resident kernels, with the indices of
// the records the encode kernel fills (rotations and maps).
struct DevStreamBuf {
    std::vector<Rec> host;
    std::vector<int32_t> enc;
    // a long stream is built as two pieces at once: the second piece (its
    // encoded positions already offset) is uploaded right behind the first
    std::vector<Rec> tail;
    std::vector<int32_t> tail_enc;
    Rec *dev = nullptr;
    const int32_t *enc_dev = nullptr;
    int n_chunks = 0;
};

// A plan uploaded to the device: one buffer holding passes, ops, maps, map
// gate indices, raw gates, the slot CSR and (resident plans) the forward and
// backward instruction streams.
struct DevPlan {
    HostPlan host;
    int host_n = 0;                  // qubits of the plan
    bool streams = false;
    DevStreamBuf sf, sb;
    // split resident streams (see split_resident): forward passes [0, split)
    // and [split, P), backward passes [split, P) and (gradient plans) [0, split);
    // split < 0: none
    DevStreamBuf h1, h2, h2b, h1b;
    int split = -1;
    // n <= 3, long plans: K >= 3 forward parts, part k = passes [cuts[k], cuts[k+1])
    // (the generators, rho_0 and <O> through the chain of the parts' transfer
    // matrices); empty otherwise
    std::vector<DevStreamBuf> parts;
    std::vector<int> cuts;
    std::vector<DevStreamBuf *> all_streams() {
        std::vector<DevStreamBuf *> v = {&sf, &sb, &h1, &h2, &h2b, &h1b};
        for (DevStreamBuf &p : parts) v.push_back(&p);
        return v;
    }
    DevBuf buf;
    Program prog{};
    const int32_t *map_gate_idx = nullptr;
    const RawGate *raw = nullptr;
    const int32_t *param_ptr = nullptr;
    const int32_t *param_rot = nullptr;
    bool built = false;
    bool encoded = false;
};

// A captured sequence of streamed launches, valid while its key is unchanged.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> key;
    std::vector<const void *> seen;  // key of the last run made without a graph
    int64_t launches = 0;            // kernels in the graph
    void *result = nullptr;          // buffer that ends up holding the result
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
        seen.clear();
        launches = 0;
        result = nullptr;
    }
};

}  // namespace

struct stab_ctx {
    int n = 0;
    int device = 0;
    int kernel = STAB_KERNEL_AUTO;
    int fuse = 1;
    stab_path_choice choice{};         // AUTO: the path tuner's choice for this n and GPU
    cudaStream_t st = nullptr;
    cudaStream_t aux = nullptr;
    cudaStream_t aux2 = nullptr;       // second branch of the split adjoint
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool own_st = false;
    cudaEvent_t ev_ready = nullptr;    // plan uploaded and encoded (on st); the aux work waits
                                       // on it (the observable's terms are uploaded on aux)
    cudaEvent_t ev_aux = nullptr;      // aux work done
    cudaEvent_t ev_stage = nullptr;    // staging buffer free
    stab_alloc_fn alloc = nullptr;
    stab_free_fn free = nullptr;
    void *user = nullptr;

    bool loaded = false;
    bool gens_valid = false;
    std::vector<stab_gate> gates;
    int64_t n_params = 0;

    DevPlan fwd, grad;
    DevBuf thetas, gens, gens_tmp, lam, rho, tmp, tmp2, terms, scal, grad_rot, partials, grads;
    DevBuf gbuf;                     // gradients written inside captured graphs
    DevBuf lam2, tmp3;               // second-branch buffers of the split sweeps
    DevBuf dotbuf;                   // partial sums of the split expectation's inner product
    DevBuf gmid;                     // split resident adjoint: rho, then lambda, at the cut
    DevBuf odense;                   // O as a dense vector, and a second vector for the
                                     // transposed products of the aligned gradient
    bool grad_aligned = false;       // the gradient plan's parts end where the generators' do
    std::vector<int> grad_cuts;      // their pass boundaries in the gradient plan (K + 1)
    DevBuf gpairs, gparts;           // the pairs at the cuts; the parts' descriptors
    std::vector<AdjPart> gparts_host;
    DevBuf chainbuf, chainbuf_e;     // n = 4 chain of transfer matrices: intermediate vectors
                                     // of the context stream's products, of <O>'s (aux)
    // split resident sweeps (n <= 6; see split_units): transfer matrix of the
    // second part (n <= 4), first-part generators, meeting vectors, basis
    // terms, batch units (generators; expectation), unit counters
    DevBuf tmat, avec, rmid, lmid, bterms, units_g, units_e, cnt;
    std::vector<const void *> key_g, key_e;
    int n_units_g = 0;
    size_t split_smem = 0;
    int sms = 0;                     // SMs of the device
    // the split sweep's launch (first-part vectors, columns of T) was made for
    // these angles when tx_gen == param_gen; ev_tx marks its end on st
    int64_t param_gen = 0, tx_gen = -1;
    cudaEvent_t ev_tx = nullptr;
    DevBuf status;                   // int32 set by kernels whose bounded waits gave up
    GraphCache g_gens, g_expect, g_grad; // streamed launch sequences (n > resident sizes)
    int64_t plan_gen = 0;            // bumped whenever a plan is rebuilt
    int32_t n_obs_terms = 0;
    bool obs_loaded = false;
    int64_t h2d_bytes = 0, d2h_bytes = 0;
    double *gens_cur = nullptr;      // buffer holding the evolved generators

    void *stage = nullptr;           // pinned host staging
    size_t stage_bytes = 0;
    void *aux_stage = nullptr;
    size_t aux_stage_bytes = 0;
    int64_t launches = 0;

    int dalloc(DevBuf &b, size_t bytes, cudaStream_t s) {
        if (b.bytes >= bytes && b.p) return STAB_OK;
        dfree(b, s);
        bytes = align256(bytes ? bytes : 256);
        void *p = nullptr;
        if (alloc) {
            p = alloc(bytes, (void *)s, user);
            if (!p) return STAB_E_NOMEM;
        } else {
            cudaError_t e = cudaMallocAsync(&p, bytes, s);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                return e == cudaErrorMemoryAllocation ? STAB_E_NOMEM : (g_last_cuda = (int)e, STAB_E_CUDA);
            }
        }
        b.p = p;
        b.bytes = bytes;
        return STAB_OK;
    }
    void dfree(DevBuf &b, cudaStream_t s) {
        if (!b.p) return;
        // a buffer may be in use on either stream of the context
        if (st) cudaStreamSynchronize(st);
        if (aux) cudaStreamSynchronize(aux);
        if (aux2) cudaStreamSynchronize(aux2);
        if (free) free(b.p, b.bytes, (void *)s, user);
        else cudaFreeAsync(b.p, s);
        b.p = nullptr;
        b.bytes = 0;
    }
    int host_stage(void *&buf, size_t &cap, size_t bytes) {
        if (cap >= bytes && buf) return STAB_OK;
        if (buf) cudaFreeHost(buf);
        buf = nullptr;
        cap = 0;
        CK(cudaMallocHost(&buf, bytes));
        cap = bytes;
        return STAB_OK;
    }
    size_t vec_bytes() const { return (sizeof(double) << (2 * n)); }
    bool use_resident() const {
        const bool k = kernel == STAB_KERNEL_AUTO ? choice.resident != 0
                                                  : (kernel == STAB_KERNEL_RESIDENT ||
                                                     kernel == STAB_KERNEL_PLAIN);
        return k && n <= kMaxResidentQubits;
    }
    bool use_resident_adjoint() const {
        const bool k = kernel == STAB_KERNEL_AUTO ? choice.resident_adjoint != 0
                                                  : kernel == STAB_KERNEL_RESIDENT;
        return k && n <= kMaxResidentAdjoint;
    }
    PlanMode fwd_mode() const {
        const bool rows = use_resident() && resident_lanes_per_group(n) == 4;
        if (kernel == STAB_KERNEL_PLAIN || !fuse) return rows ? PLAN_PLAIN_ROWS : PLAN_PLAIN;
        return rows ? PLAN_ROWS : PLAN_FUSED;
    }
};

namespace {

// Uploads a host plan into its device buffer (one copy from pinned staging).
int upload_plan(stab_ctx *c, DevPlan &P) {
    HostPlan &H = P.host;
    // resident plans read only their streams (plus maps and raw gates for encoding)
    const size_t n_pass = P.streams ? 0 : H.passes.size();
    const size_t n_ops = P.streams ? 0 : H.ops.size();
    const size_t b_pass = align256(n_pass * sizeof(DevPass));
    const size_t b_ops = align256(n_ops * sizeof(DevOp));
    const size_t b_maps = align256(H.maps.size() * sizeof(DevMap3));
    const size_t b_midx = align256(H.map_gate_idx.size() * sizeof(int32_t));
    const size_t b_raw = align256(H.raw.size() * sizeof(RawGate));
    const size_t b_pptr = align256(H.param_ptr.size() * sizeof(int32_t));
    const size_t b_prot = align256(H.param_rot.size() * sizeof(int32_t));
    const size_t b_tabs = align256(H.tabs.size() * sizeof(DevTab));
    const std::vector<DevStreamBuf *> streams = P.all_streams();
    size_t b_streams = 0;
    for (const DevStreamBuf *S : streams)
        b_streams += align256((S->host.size() + S->tail.size()) * sizeof(Rec)) +
                     align256((S->enc.size() + S->tail_enc.size()) * 4);
    const size_t total = b_pass + b_ops + b_maps + b_midx + b_raw + b_pptr + b_prot + b_tabs +
                         b_streams;
    RC(c->dalloc(P.buf, total, c->st));
    CK(cudaEventSynchronize(c->ev_stage));
    RC(c->host_stage(c->stage, c->stage_bytes, total));
    char *h = (char *)c->stage;
    char *d = (char *)P.buf.p;
    size_t off = 0;
    // large pieces are copied into the staging buffer by the host pool
    std::vector<std::function<void()>> copies;
    // [src, bytes) then [src2, bytes2) at the next `span` bytes of the buffer
    auto put = [&](const void *src, size_t bytes, size_t span, const void *src2 = nullptr,
                   size_t bytes2 = 0) {
        size_t o = off;
        for (int k = 0; k < 2; ++k) {
            const void *from = k ? src2 : src;
            const size_t b = k ? bytes2 : bytes;
            if (b >= ((size_t)1 << 18)) {
                char *dst = h + o;
                copies.push_back([dst, from, b] { std::memcpy(dst, from, b); });
            } else if (b) {
                std::memcpy(h + o, from, b);
            }
            o += b;
        }
        const size_t at = off;
        off += span;
        return d + at;
    };
    P.prog.passes = (const DevPass *)put(H.passes.data(), n_pass * sizeof(DevPass), b_pass);
    P.prog.ops = (const DevOp *)put(H.ops.data(), n_ops * sizeof(DevOp), b_ops);
    P.prog.maps = (const DevMap3 *)put(H.maps.data(), H.maps.size() * sizeof(DevMap3), b_maps);
    P.map_gate_idx = (const int32_t *)put(H.map_gate_idx.data(), H.map_gate_idx.size() * 4, b_midx);
    P.raw = (const RawGate *)put(H.raw.data(), H.raw.size() * sizeof(RawGate), b_raw);
    P.param_ptr = (const int32_t *)put(H.param_ptr.data(), H.param_ptr.size() * 4, b_pptr);
    P.param_rot = (const int32_t *)put(H.param_rot.data(), H.param_rot.size() * 4, b_prot);
    P.prog.tabs = (const DevTab *)put(H.tabs.data(), H.tabs.size() * sizeof(DevTab), b_tabs);
    for (DevStreamBuf *S : streams) {
        const size_t rb = S->host.size() * sizeof(Rec), tb = S->tail.size() * sizeof(Rec);
        S->dev = (Rec *)put(S->host.data(), rb, align256(rb + tb), S->tail.data(), tb);
        const size_t eb = S->enc.size() * 4, teb = S->tail_enc.size() * 4;
        S->enc_dev = (const int32_t *)put(S->enc.data(), eb, align256(eb + teb),
                                          S->tail_enc.data(), teb);
    }
    P.prog.n_passes = (int32_t)n_pass;
    P.prog.n_ops = (int32_t)n_ops;
    HostPool::run(copies);
    CK(cudaMemcpyAsync(P.buf.p, h, total, cudaMemcpyHostToDevice, c->st));
    CK(cudaEventRecord(c->ev_stage, c->st));
    c->h2d_bytes += (int64_t)total;
    P.built = true;
    P.encoded = false;
    return STAB_OK;
}

int encode_plan(stab_ctx *c, DevPlan &P) {
    const double *th = (const double *)c->thetas.p;
    if (P.streams) {
        // resident plans: only the instruction streams are read by kernels;
        // each run's map is composed once and copied into every stream
        const int n_maps = (int)P.host.maps.size();
        if (n_maps > 0) {
            CK(launch_compose_maps(const_cast<DevMap3 *>(P.prog.maps), n_maps,
                                   max_map_count(P.host.maps.data(), P.host.maps.size()),
                                   P.map_gate_idx, P.raw, th, c->st));
            c->launches++;
        }
        for (DevStreamBuf *S : P.all_streams()) {
            const int n_enc = (int)(S->enc.size() + S->tail_enc.size());
            if (n_enc == 0) continue;
            CK(launch_encode_stream(S->dev, S->enc_dev, n_enc, P.prog.maps, th,
                                    c->st));
            c->launches++;
        }
        P.encoded = true;
        return STAB_OK;
    }
    const int n_ops = P.prog.n_ops, n_maps = (int)P.host.maps.size();
    if (n_ops == 0 && n_maps == 0) {
        P.encoded = true;
        return STAB_OK;
    }
    CK(launch_encode(const_cast<DevOp *>(P.prog.ops), n_ops, const_cast<DevMap3 *>(P.prog.maps),
                     n_maps, max_map_count(P.host.maps.data(), P.host.maps.size()),
                     P.map_gate_idx, P.raw, th, c->st));
    c->launches += (n_maps > 0) + (n_ops > 0);
    P.encoded = true;
    return STAB_OK;
}

// One instruction stream to build: passes [k0, k1) of the plan, forward or
// (backward) walked from k1 - 1 down to k0.
struct StreamSpec {
    DevStreamBuf *S;
    bool backward;
    int k0, k1;
};

// Streams of at least this many passes are built as two pieces at once.
constexpr int kStreamPiecePasses = 4096;

// Builds the streams, on the host pool when `threads` is set; there a long
// stream is built as two pieces at once, the first ending in R_NEXT on a
// chunk boundary (its pending pulls in an identity pass), the second in
// S.tail -- the same passes, pulls and ops as the one-piece stream.
void build_streams(const DevPlan &P, const std::vector<StreamSpec> &specs, bool threads) {
    std::vector<std::function<void()>> jobs;
    for (const StreamSpec &sp : specs) {
        DevStreamBuf *S = sp.S;
        S->tail.clear();
        S->tail_enc.clear();
        if (!threads || sp.k1 - sp.k0 < kStreamPiecePasses) {
            jobs.push_back([&P, sp] {
                build_stream(P.host, sp.backward, &sp.S->host, sp.k0, sp.k1, &sp.S->enc);
            });
            continue;
        }
        const int mid = sp.k0 + (sp.k1 - sp.k0) / 2;
        const int a0 = sp.backward ? mid : sp.k0, a1 = sp.backward ? sp.k1 : mid;
        const int b0 = sp.backward ? sp.k0 : mid, b1 = sp.backward ? mid : sp.k1;
        jobs.push_back([&P, sp, a0, a1] {
            build_stream(P.host, sp.backward, &sp.S->host, a0, a1, &sp.S->enc, false);
        });
        jobs.push_back([&P, sp, b0, b1] {
            build_stream(P.host, sp.backward, &sp.S->tail, b0, b1, &sp.S->tail_enc);
        });
    }
    if (threads) {
        HostPool::run(jobs);
    } else {
        for (auto &j : jobs) j();
    }
    for (const StreamSpec &sp : specs) {
        DevStreamBuf &S = *sp.S;
        for (int32_t &e : S.tail_enc) e += (int32_t)S.host.size();
        S.n_chunks = (int)((S.host.size() + S.tail.size()) / kChunkRecs);
    }
}

// Forward and backward streams, built concurrently on host threads; with
// split_frac > 0 (and enough passes) also the split streams cut at that
// fraction of the passes.  A split gradient plan (grad) needs only the four
// half streams, not the whole-circuit ones.  Below kThreadedStreamPasses
// passes the streams are built on the calling thread: handing them to the
// pool would cost more than the work.
void make_streams(DevPlan &P, double split_frac = 0.0, bool grad = false, int n_parts = 2,
                  double first_frac = 0.0, int force_split = -1) {
    P.streams = true;
    const int np = (int)P.host.passes.size();
    const bool threads = np >= kThreadedStreamPasses;
    if (!grad && n_parts >= 3) {
        // K forward parts of equal pass counts, or (first_frac > 0) a first
        // part of that fraction of the passes and K - 1 equal parts after it
        P.sf = P.sb = P.h1 = P.h2 = P.h2b = P.h1b = DevStreamBuf();
        P.parts.resize((size_t)n_parts);
        P.cuts.assign((size_t)n_parts + 1, 0);
        if (first_frac > 0.0) {
            const int c1 = (int)(np * first_frac);
            for (int k = 1; k <= n_parts; ++k)
                P.cuts[k] = c1 + (int)((int64_t)(np - c1) * (k - 1) / (n_parts - 1));
        } else {
            for (int k = 0; k <= n_parts; ++k) P.cuts[k] = (int)((int64_t)np * k / n_parts);
        }
        P.split = P.cuts[1];
        std::vector<StreamSpec> specs;
        for (int k = 0; k < n_parts; ++k)
            specs.push_back({&P.parts[k], false, P.cuts[k], P.cuts[k + 1]});
        build_streams(P, specs, threads);
        return;
    }
    P.parts.clear();
    P.cuts.clear();
    P.split = (split_frac > 0.0 && np >= kSplitMinPasses) ? (int)(np * split_frac) : -1;
    if (P.split >= 0 && force_split > 0 && force_split < np) P.split = force_split;
    // streams that are rebuilt keep their capacity; the others are released
    if (P.split < 0) P.h1 = P.h2 = P.h2b = DevStreamBuf();
    if (!(grad && P.split >= 0)) P.h1b = DevStreamBuf();
    if (grad && P.split >= 0) {
        P.sf = P.sb = DevStreamBuf();
        build_streams(P,
                      {{&P.h1b, true, 0, P.split},
                       {&P.h1, false, 0, P.split},
                       {&P.h2, false, P.split, np},
                       {&P.h2b, true, P.split, np}},
                      threads);
        return;
    }
    if (P.split < 0) {
        build_streams(P, {{&P.sf, false, 0, np}, {&P.sb, true, 0, np}}, threads);
        return;
    }
    // A split plan reads the halves: the generators (n <= 4) and the density
    // matrix through h1 and h2, <O> through h1 and h2b.  Only n = 5, 6 still
    // read the whole forward stream (their generators and density matrix are
    // not split); nothing reads the whole backward stream.
    P.sb = DevStreamBuf();
    const bool whole_fwd = P.host_n > 4;
    if (!whole_fwd) P.sf = DevStreamBuf();
    std::vector<StreamSpec> specs = {
        {&P.h1, false, 0, P.split}, {&P.h2, false, P.split, np}, {&P.h2b, true, P.split, np}};
    if (whole_fwd) specs.push_back({&P.sf, false, 0, np});
    build_streams(P, specs, threads);
}

// Gradient streams of a many-part split at the pass boundaries `cuts` (K + 1
// of them, 0 and P included): part 0 backward over [0, cuts[1]) (walked from
// its end), part k >= 1 forward over [cuts[k], cuts[k + 1]).
void make_grad_part_streams(DevPlan &P, const std::vector<int> &cuts) {
    P.streams = true;
    const int np = (int)P.host.passes.size();
    const size_t K = cuts.size() - 1;
    P.sf = P.sb = P.h1 = P.h2 = P.h2b = P.h1b = DevStreamBuf();
    P.parts.resize(K);
    P.cuts = cuts;
    P.split = cuts[1];
    std::vector<StreamSpec> specs;
    for (size_t k = 0; k < K; ++k)
        specs.push_back({&P.parts[k], k == 0, cuts[k], cuts[k + 1]});
    build_streams(P, specs, np >= kThreadedStreamPasses);
}

void no_streams(DevPlan &P) {
    P.streams = false;
    P.sf = DevStreamBuf();
    P.sb = DevStreamBuf();
    P.h1 = P.h2 = P.h2b = P.h1b = DevStreamBuf();
    P.parts.clear();
    P.cuts.clear();
    P.split = -1;
}

// Reads and clears the kernels' status word (synchronizes the context).
int check_status(stab_ctx *c) {
    if (!c->status.p) return STAB_OK;
    int32_t h = 0;
    CK(cudaStreamSynchronize(c->aux));
    CK(cudaMemcpyAsync(&h, c->status.p, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (h != 0) {
        CK(cudaMemsetAsync(c->status.p, 0, sizeof(int32_t), c->st));
        CK(cudaStreamSynchronize(c->st));
        return STAB_E_TIMEOUT;
    }
    return STAB_OK;
}

int upload_thetas_host(stab_ctx *c, const double *thetas) {
    const size_t bytes = (size_t)(c->n_params > 0 ? c->n_params : 1) * sizeof(double);
    RC(c->dalloc(c->thetas, bytes, c->st));
    if (c->n_params == 0) return STAB_OK;
    CK(cudaEventSynchronize(c->ev_stage));
    RC(c->host_stage(c->stage, c->stage_bytes, bytes));
    std::memcpy(c->stage, thetas, (size_t)c->n_params * sizeof(double));
    CK(cudaMemcpyAsync(c->thetas.p, c->stage, (size_t)c->n_params * sizeof(double),
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaEventRecord(c->ev_stage, c->st));
    c->h2d_bytes += c->n_params * (int64_t)sizeof(double);
    return STAB_OK;
}

// Uploads deduplicated observable terms on the main stream (pinned staging).
int upload_terms(stab_ctx *c, const stab_term *O, int64_t n_terms) {
    std::vector<DevTerm> t;
    RC(encode_terms(c->n, O, n_terms, &t));
    const size_t bytes = (t.size() ? t.size() : 1) * sizeof(DevTerm);
    // The terms are read on the aux stream (expectations, gradients), so they
    // are uploaded there, from the aux staging buffer: the upload does not
    // queue behind generator work on the main stream.  The aux stream may
    // still read the previous terms and its staging buffer.
    CK(cudaStreamSynchronize(c->aux));
    RC(c->dalloc(c->terms, bytes, c->aux));
    if (!t.empty()) {
        RC(c->host_stage(c->aux_stage, c->aux_stage_bytes, bytes));
        std::memcpy(c->aux_stage, t.data(), t.size() * sizeof(DevTerm));
        CK(cudaMemcpyAsync(c->terms.p, c->aux_stage, t.size() * sizeof(DevTerm),
                           cudaMemcpyHostToDevice, c->aux));
        c->h2d_bytes += (int64_t)(t.size() * sizeof(DevTerm));
    }
    c->n_obs_terms = (int32_t)t.size();
    return STAB_OK;
}

void bit_runs(const std::vector<int> &bits, BitRuns *r) {
    // bit k of a packed integer goes to index bit bits[k] (bits ascending)
    std::memset(r, 0, sizeof(*r));
    for (size_t k = 0; k < bits.size();) {
        size_t j = k + 1;
        while (j < bits.size() && bits[j] == bits[j - 1] + 1) ++j;
        r->src[r->n] = (uint8_t)k;
        r->dst[r->n] = (uint8_t)bits[k];
        r->len[r->n] = (uint8_t)(j - k);
        r->n++;
        k = j;
    }
}

// Tile geometry for wire passes on `wires`: the wires' x and z bits plus as
// many of the lowest other bits as keep at least 256 tiles (and 4096 entries).
void make_tile_group(int n, int n_vec, const std::vector<const DevPass *> &group, int inverse,
                     TileGroup *tg, int min_tiles = 256, int max_bits = kTileMaxBits) {
    std::memset(tg, 0, sizeof(*tg));
    std::vector<int> wires;
    for (const DevPass *p : group)
        if (std::find(wires.begin(), wires.end(), (int)p->q) == wires.end()) wires.push_back(p->q);
    std::vector<int> qbits;
    for (int q : wires) {
        qbits.push_back(q);
        qbits.push_back(n + q);
    }
    std::vector<int> others;
    for (int b = 0; b < 2 * n; ++b)
        if (std::find(qbits.begin(), qbits.end(), b) == qbits.end()) others.push_back(b);
    int c = 0;
    while (c < (int)others.size() && (int)qbits.size() + c + 1 <= max_bits &&
           ((int64_t)n_vec << (2 * n - ((int)qbits.size() + c + 1))) >= min_tiles)
        ++c;
    std::vector<int> tile(qbits);
    tile.insert(tile.end(), others.begin(), others.begin() + c);
    std::sort(tile.begin(), tile.end());
    std::vector<int> rest(others.begin() + c, others.end());
    tg->n_pass = (int32_t)group.size();
    tg->tile_bits = (int32_t)tile.size();
    tg->rest_bits = (int32_t)rest.size();
    tg->inverse = inverse;
    for (size_t j = 0; j < group.size(); ++j) {
        const int q = group[j]->q;
        tg->lz[j] = (uint8_t)(std::find(tile.begin(), tile.end(), q) - tile.begin());
        tg->lx[j] = (uint8_t)(std::find(tile.begin(), tile.end(), n + q) - tile.begin());
        tg->n_ops[j] = group[j]->n_ops;
        tg->first[j] = group[j]->first;
    }
    bit_runs(tile, &tg->tile_runs);
    bit_runs(rest, &tg->rest_runs);
}

// ---------------------------------------------------------------- split resident sweeps
//
// A resident vector walks the circuit's passes one after another on one SM.
// With the passes cut at `split` (DevPlan h1 = [0, split), h2 = [split, P)):
//   generators (n <= 4): U Z_k U^dagger = T a_k with a_k = Z_k through h1 and
//     T the transfer matrix of h2, whose 4^n - 1 nontrivial columns are the
//     basis strings through h2 -- 4^n - 1 + n independent vectors, one batch
//     launch, then one product;
//   <O> = <lambda, r> with r = rho_0 through h1 and lambda = O backward through
//     h2 -- two vectors at once, then one inner product.
// Every part runs on its own CTA of the persistent batch kernel, except the
// columns of T at n = 4 (255 of them, more than the SMs): k_transfer_cols
// carries them two to a CTA.

bool split_gens_ok(const stab_ctx *c) { return c->fwd.split >= 0 && c->n <= 4; }

// n <= 3: parts of a long plan for the chain of transfer matrices -- as many
// as the SMs hold one unit each (n generators and rho_0 through the first
// part, 4^n - 1 columns per further part, two CTAs left for other work),
// each part at least kChainMinPasses passes; < 3 means the two-part split.
constexpr int kChainMinPasses = 32;
int chain_parts(const stab_ctx *c) {
    if (c->n > 3) return 2;
    const int E = 1 << (2 * c->n);
    const int np = (int)c->fwd.host.passes.size();
    const int by_sms = 1 + (c->sms - (c->n + 1) - 2) / (E - 1);
    const int by_len = np / kChainMinPasses;
    const int k = std::min(by_sms, by_len);
    return k >= 3 ? k : 2;
}

bool chain_mode(const stab_ctx *c) { return !c->fwd.parts.empty(); }
bool split_expect_ok(const stab_ctx *c) { return c->fwd.split >= 0; }

int split_setup(stab_ctx *c, cudaStream_t s) {
    if (c->split_smem == 0) {
        // n = 4: as much shared memory as a k_transfer_cols CTA takes, so a
        // first-part unit (the critical path) never shares an SM's FP64 pipe
        // with a CTA of columns running beside it
        c->split_smem = transfer_cols_ctas(c->n) > 0
                            ? std::max(batch_smem_bytes(c->n), transfer_cols_smem())
                            : batch_smem_bytes(c->n);
        int occ = 0;
        CK(batch_occupancy(c->split_smem, &occ));
    }
    const int E = 1 << (2 * c->n);
    RC(c->dalloc(c->cnt, 256, s));
    RC(c->dalloc(c->rmid, (size_t)E * 8, s));
    RC(c->dalloc(c->lmid, (size_t)E * 8, s));
    RC(c->dalloc(c->dotbuf, 256 * sizeof(double), s));
    return STAB_OK;
}

// Units of the generators' split sweep (rebuilt when the plan changes):
// the first part carries Z_0 .. Z_{n-1} and rho_0 into avec, the second part
// the basis strings into the columns of T.
int split_units_g(stab_ctx *c) {
    const int n = c->n, E = 1 << (2 * n);
    // one transfer matrix per part after the first
    const int n_mats = chain_mode(c) ? (int)c->fwd.parts.size() - 1 : 1;
    RC(split_setup(c, c->st));
    RC(c->dalloc(c->tmat, (size_t)n_mats * E * E * 8, c->st));
    RC(c->dalloc(c->avec, (size_t)(n + 1) * E * 8, c->st));
    RC(c->dalloc(c->bterms, (size_t)E * sizeof(DevTerm), c->st));
    RC(c->dalloc(c->units_g, (size_t)(n_mats * (E - 1) + n + 1) * sizeof(BatchUnit), c->st));
    const DevStreamBuf &first = chain_mode(c) ? c->fwd.parts[0] : c->fwd.h1;
    const std::vector<const void *> key = {(const void *)c->plan_gen, first.dev,
                                           c->fwd.h2.dev, c->tmat.p, c->avec.p, c->bterms.p,
                                           c->units_g.p, (const void *)(intptr_t)n_mats};
    if (key == c->key_g) return STAB_OK;
    std::vector<BatchUnit> U;
    for (int k = 0; k < n; ++k) {
        BatchUnit u{};
        u.stream = first.dev;
        u.n_chunks = first.n_chunks;
        u.n = (int8_t)n;
        u.init = INIT_GENERATOR;
        u.gen = (int16_t)k;
        u.out = (double *)c->avec.p + (size_t)k * E;
        U.push_back(u);
    }
    {
        // rho_0 through the first part, for the density matrix (r = T r_1)
        BatchUnit u{};
        u.stream = first.dev;
        u.n_chunks = first.n_chunks;
        u.n = (int8_t)n;
        u.init = INIT_RHO0;
        u.out = (double *)c->avec.p + (size_t)n * E;
        U.push_back(u);
    }
    // the columns of T: units of the same launch, or (n = 4, where they would
    // outnumber the SMs) the two-column CTAs of k_transfer_cols
    const int n_basis = transfer_cols_ctas(n) > 0 ? 1 : E;
    std::vector<DevTerm> basis((size_t)E);
    for (int j = 1; j < E; ++j) basis[(size_t)j] = DevTerm{1.0, (uint64_t)j};
    for (int mtx = 0; mtx < n_mats; ++mtx) {
        const DevStreamBuf &part = chain_mode(c) ? c->fwd.parts[(size_t)mtx + 1] : c->fwd.h2;
        for (int j = 1; j < n_basis; ++j) {
            BatchUnit u{};
            u.stream = part.dev;
            u.n_chunks = part.n_chunks;
            u.n = (int8_t)n;
            u.init = INIT_TERMS;
            u.terms = (const DevTerm *)c->bterms.p + j;
            u.n_terms = 1;
            u.out = (double *)c->tmat.p + (size_t)mtx * E * E + (size_t)j * E;
            U.push_back(u);
        }
    }
    // column 0 of every T: the identity string stays itself
    std::vector<double> col0((size_t)E, 0.0);
    col0[0] = 1.0;
    for (int mtx = 0; mtx < n_mats; ++mtx)
        CK(cudaMemcpyAsync((double *)c->tmat.p + (size_t)mtx * E * E, col0.data(), (size_t)E * 8,
                           cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->bterms.p, basis.data(), basis.size() * sizeof(DevTerm),
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->units_g.p, U.data(), U.size() * sizeof(BatchUnit),
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));   // the host vectors above are temporaries
    c->n_units_g = (int)U.size();
    c->key_g = key;
    return STAB_OK;
}

// The generators' split sweep on the context stream: the first-part vectors
// into avec and the columns of T into tmat (the caller applies T).
int split_run_g(stab_ctx *c) {
    RC(split_units_g(c));
    BatchArgs a{};
    a.units = (const BatchUnit *)c->units_g.p;
    a.n_units = c->n_units_g;
    a.counter = (int32_t *)c->cnt.p;
    a.status = (int32_t *)c->status.p;
    CK(cudaMemsetAsync(c->cnt.p, 0, 4, c->st));
    if (transfer_cols_ctas(c->n) > 0) {
        // the first-part units and the columns of T (of both later parts in
        // a three-part chain) at once, on two streams
        CK(cudaEventRecord(c->ev_fork, c->st));
        CK(cudaStreamWaitEvent(c->aux2, c->ev_fork, 0));
        CK(launch_batch(a, c->n_units_g, c->split_smem, c->st));
        ColArgs ca{};
        if (chain_mode(c)) {
            ca.n_parts = (int)c->fwd.parts.size() - 1;
            if (ca.n_parts > 2) return STAB_E_STATE;
            for (int k = 0; k < ca.n_parts; ++k) {
                ca.stream[k] = c->fwd.parts[(size_t)k + 1].dev;
                ca.n_chunks[k] = c->fwd.parts[(size_t)k + 1].n_chunks;
            }
        } else {
            ca.n_parts = 1;
            ca.stream[0] = c->fwd.h2.dev;
            ca.n_chunks[0] = c->fwd.h2.n_chunks;
        }
        ca.tmat = (double *)c->tmat.p;
        ca.status = (int32_t *)c->status.p;
        CK(launch_transfer_cols(ca, c->n, c->aux2));
        CK(cudaEventRecord(c->ev_join, c->aux2));
        CK(cudaStreamWaitEvent(c->st, c->ev_join, 0));
        c->launches++;
    } else {
        CK(launch_batch(a, c->n_units_g, c->split_smem, c->st));
    }
    c->launches++;
    CK(cudaEventRecord(c->ev_tx, c->st));
    c->tx_gen = c->param_gen;
    return STAB_OK;
}

// Applies the chain of the parts' transfer matrices (chain mode) or the one
// transfer matrix to n_vec first-part vectors of avec starting at `first`.
int split_apply(stab_ctx *c, int first, int n_vec, double *out, const DevTerm *terms, int n_terms,
                double *dot_out, cudaStream_t s) {
    const size_t E = (size_t)1 << (2 * c->n);
    const double *in = (const double *)c->avec.p + (size_t)first * E;
    if (chain_mode(c) && transfer_cols_ctas(c->n) > 0) {
        // n = 4: one matrix-vector product per part, through a scratch pair
        // of the calling stream's own (<O> on aux may overlap the generators)
        DevBuf &scratch = s == c->st ? c->chainbuf : c->chainbuf_e;
        RC(c->dalloc(scratch, 2 * (size_t)n_vec * E * 8, s));
        const int n_mats = (int)c->fwd.parts.size() - 1;
        CK(launch_apply_transfer_chain((const double *)c->tmat.p, n_mats, in, out,
                                       (double *)scratch.p, n_vec, c->n, terms, n_terms, dot_out,
                                       s));
        c->launches += n_mats + (dot_out ? 1 : 0);   // a product per matrix, then the dot
    } else if (chain_mode(c)) {
        CK(launch_apply_chain((const double *)c->tmat.p, (int)c->fwd.parts.size() - 1, in, out,
                              n_vec, c->n, terms, n_terms, dot_out, s));
        c->launches++;
    } else {
        CK(launch_apply_transfer((const double *)c->tmat.p, in, out, n_vec, c->n, s));
        c->launches++;
    }
    return STAB_OK;
}

// Units of the expectation's split sweep on stream s (rebuilt when the plan
// or the observable's device terms change).
int split_units_e(stab_ctx *c, cudaStream_t s) {
    RC(split_setup(c, s));
    RC(c->dalloc(c->units_e, 2 * sizeof(BatchUnit), s));
    const int32_t nt = c->n_obs_terms;
    const std::vector<const void *> key = {(const void *)c->plan_gen, c->fwd.h1.dev,
                                           c->fwd.h2b.dev, c->terms.p, (const void *)(intptr_t)nt,
                                           c->rmid.p, c->lmid.p, c->units_e.p};
    if (key == c->key_e) return STAB_OK;
    BatchUnit U[2] = {};
    U[0].stream = c->fwd.h1.dev;
    U[0].n_chunks = c->fwd.h1.n_chunks;
    U[0].n = (int8_t)c->n;
    U[0].init = INIT_RHO0;
    U[0].out = (double *)c->rmid.p;
    U[1].stream = c->fwd.h2b.dev;
    U[1].n_chunks = c->fwd.h2b.n_chunks;
    U[1].n = (int8_t)c->n;
    U[1].init = INIT_TERMS;
    U[1].terms = (const DevTerm *)c->terms.p;
    U[1].n_terms = nt;
    U[1].out = (double *)c->lmid.p;
    CK(cudaMemcpyAsync(c->units_e.p, U, sizeof(U), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    c->key_e = key;
    return STAB_OK;
}

// Streamed propagation of n_vec vectors through a plan; *cur / *alt are the
// ping-pong buffers (the result ends in *cur).  Consecutive wire passes on at
// most kTileWires wires run as one tile-fused launch (fused plans only; the
// gate-by-gate forms keep one launch per gate).
int run_streamed(stab_ctx *c, const DevPlan &P, double **cur, double **alt, int n_vec,
                 int inverse, cudaStream_t s, int k0 = 0, int k1 = -1) {
    const auto &passes = P.host.passes;
    if (k1 < 0) k1 = (int)passes.size();
    const int np = k1 - k0;   // passes [k0, k1), walked backward when inverse
    // tiles pay where a launch is small (launch-bound: few vectors, n <= 8); larger
    // launches are FP64-bound and run faster one wire per launch; the limit is
    // the path tuner's (measured per GPU model)
    const bool fuse_tiles = P.host.mode != PLAN_PLAIN && P.host.mode != PLAN_PLAIN_ROWS &&
                            ((uint64_t)n_vec << (2 * c->n)) <= (uint64_t)c->choice.tile_limit;
    std::vector<const DevPass *> group;
    std::vector<int> wires;
    // with tiles, a Clifford gather is folded into the loads of the next group
    const DevPass *pending = nullptr;
    auto gather_now = [&]() -> int {
        CK(launch_stream_cliff(*cur, *alt, c->n, n_vec, *pending, P.prog.ops, inverse, s));
        std::swap(*cur, *alt);
        c->launches++;
        pending = nullptr;
        return STAB_OK;
    };
    auto flush = [&]() -> int {
        if (group.empty()) return STAB_OK;
        if (group.size() == 1 && !pending) {
            CK(launch_stream_wire(*cur, c->n, n_vec, *group[0], P.prog.ops, P.prog.maps, inverse,
                                  s));
        } else {
            TileGroup tg;
            make_tile_group(c->n, n_vec, group, inverse, &tg);
            double *dst = *cur;
            if (pending) {
                tg.pull_n = pending->n_ops;
                tg.pull_first = pending->first;
                tg.pull_inverse = inverse;
                dst = *alt;
            }
            CK(launch_stream_tile(*cur, dst, c->n, n_vec, tg, P.prog.ops, P.prog.maps, s));
            if (pending) {
                std::swap(*cur, *alt);
                pending = nullptr;
            }
        }
        c->launches++;
        group.clear();
        wires.clear();
        return STAB_OK;
    };
    for (int k = 0; k < np; ++k) {
        const DevPass &p = passes[inverse ? k1 - 1 - k : k0 + k];
        if (p.type == P_WIRE) {
            const bool known = std::find(wires.begin(), wires.end(), (int)p.q) != wires.end();
            if (!fuse_tiles || (int)group.size() == kTileMaxPasses ||
                (!known && (int)wires.size() == kTileWires)) {
                RC(flush());
            }
            group.push_back(&p);
            if (std::find(wires.begin(), wires.end(), (int)p.q) == wires.end())
                wires.push_back(p.q);
            continue;
        }
        RC(flush());
        if (pending) RC(gather_now());
        if (p.type == P_TAB) {
            // a long Clifford run: one gather through its tableau
            CK(launch_stream_tab(*cur, *alt, c->n, n_vec, P.prog.tabs + 2 * p.first + (inverse ? 1 : 0),
                                 s));
            std::swap(*cur, *alt);
            c->launches++;
            continue;
        }
        pending = &p;
        if (!fuse_tiles) RC(gather_now());
    }
    RC(flush());
    if (pending) RC(gather_now());
    return STAB_OK;
}

// Replays the launch sequence `body` (queued on s) from a graph cached under
// `key`, capturing it first when the key changed.  s is the context's own
// non-blocking stream (the legacy default stream cannot be captured).  All
// buffers the body uses must be allocated before the call.
template <class F>
int run_graph(stab_ctx *c, GraphCache &g, const std::vector<const void *> &key, cudaStream_t s,
              F body) {
    if (!(g.exec && g.key == key) && g.seen != key) {
        // First run of this sequence: launched directly.  A sequence that is
        // run once (a served request, a one-off circuit) would only pay for
        // capturing and instantiating a graph; it is captured when it comes
        // again.
        if (g.exec) g.reset();
        const int rc = body(s, &g.result);
        if (rc != STAB_OK) return rc;
        g.seen = key;
        return STAB_OK;
    }
    if (!g.exec || g.key != key) {
        g.reset();
        cudaGraph_t graph = nullptr;
        const int64_t l0 = c->launches;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const int rc = body(s, &g.result);
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        g.launches = c->launches - l0;
        c->launches = l0;
        if (rc != STAB_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            g.reset();
            if (rc != STAB_OK) return rc;
            CK(e);
        }
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) g.reset();
        CK(e);
        g.key = key;
    }
    CK(cudaGraphLaunch(g.exec, s));
    c->launches += g.launches;
    return STAB_OK;
}

void reset_graphs(stab_ctx *c) {
    c->g_gens.reset();
    c->g_expect.reset();
    c->g_grad.reset();
    c->plan_gen++;
}

// Plans of one gate list in different modes hold the same sequence of units:
// a P_CLIFF pass, or a maximal stretch of consecutive P_WIRE passes on one
// wire (a gradient plan only cuts a wire's run into several passes).  Returns
// the pass of plan B that starts the unit starting at pass k of plan A, or -1
// when pass k starts no unit or the two plans' unit sequences differ (a run
// that is the identity and holds no rotation makes no pass in some modes).
bool unit_start(const HostPlan &P, size_t i) {
    if (i == 0) return true;
    const DevPass &p = P.passes[i], &q = P.passes[i - 1];
    return p.type != P_WIRE || q.type != P_WIRE || p.q != q.q;
}

int aligned_pass(const HostPlan &A, int k, const HostPlan &B) {
    if (k <= 0 || k >= (int)A.passes.size() || !unit_start(A, (size_t)k)) return -1;
    // the units of both plans, as (type, wire), in order; the first pass of each in B
    std::vector<uint16_t> ua, ub;
    std::vector<int> start_b;
    int unit_k = -1;
    for (size_t i = 0; i < A.passes.size(); ++i)
        if (unit_start(A, i)) {
            if ((int)i == k) unit_k = (int)ua.size();
            ua.push_back((uint16_t)(A.passes[i].type << 8 | A.passes[i].q));
        }
    for (size_t i = 0; i < B.passes.size(); ++i)
        if (unit_start(B, i)) {
            ub.push_back((uint16_t)(B.passes[i].type << 8 | B.passes[i].q));
            start_b.push_back((int)i);
        }
    if (ua != ub || unit_k < 0) return -1;
    return start_b[(size_t)unit_k];
}

int ensure_grad_plan(stab_ctx *c) {
    if (!c->grad.built) {
        build_plan(c->n, c->gates.data(), (int64_t)c->gates.size(), c->n_params, PLAN_GRAD,
                   &c->grad.host, !c->use_resident_adjoint());
        // resident adjoint: split at half the passes (the AUTO kernel; the
        // RESIDENT choice keeps the single-CTA forward-then-reverse sweep) --
        // or, at n = 4 with the generators' split sweep, at the gate where the
        // generators' first part ends, so the pair at the cut comes from that
        // sweep (see stab_grad_async)
        c->grad_aligned = false;
        c->grad_cuts.clear();
        if (c->use_resident_adjoint()) {
            // the generators' part boundaries, as passes of the gradient plan
            const int npg = (int)c->grad.host.passes.size();
            if (c->kernel == STAB_KERNEL_AUTO && c->use_resident() && split_gens_ok(c) &&
                npg >= kSplitMinPasses) {
                std::vector<int> fc = chain_mode(c)
                                          ? c->fwd.cuts
                                          : std::vector<int>{0, c->fwd.split,
                                                             (int)c->fwd.host.passes.size()};
                std::vector<int> gc = {0};
                for (size_t k = 1; k + 1 < fc.size(); ++k) {
                    const int g = aligned_pass(c->fwd.host, fc[k], c->grad.host);
                    if (g <= gc.back()) break;
                    gc.push_back(g);
                }
                if (gc.size() + 1 == fc.size() && gc.back() < npg) {
                    gc.push_back(npg);
                    c->grad_cuts = gc;
                }
            }
            if (!c->grad_cuts.empty()) make_grad_part_streams(c->grad, c->grad_cuts);
            else make_streams(c->grad, c->kernel == STAB_KERNEL_AUTO ? 0.5 : 0.0, true);
            c->grad_aligned = !c->grad_cuts.empty();
        } else {
            no_streams(c->grad);
        }
        c->g_grad.reset();
        c->plan_gen++;
        RC(upload_plan(c, c->grad));
        if (c->grad_aligned) {
            // the parts' descriptors: part 0 backward from the pair at the first
            // cut, part k >= 1 forward from the pair at cut k
            const int K = (int)c->grad_cuts.size() - 1;
            const size_t E = (size_t)1 << (2 * c->n);
            RC(c->dalloc(c->gpairs, (size_t)(K - 1) * 2 * E * sizeof(double), c->st));
            RC(c->dalloc(c->gparts, (size_t)K * sizeof(AdjPart), c->st));
            const double *pairs = (const double *)c->gpairs.p;
            c->gparts_host.assign((size_t)K, AdjPart{});
            for (int k = 0; k < K; ++k) {
                AdjPart &q = c->gparts_host[(size_t)k];
                const int at = k == 0 ? 1 : k;   // the pair this part starts from
                q.stream = c->grad.parts[(size_t)k].dev;
                q.n_chunks = c->grad.parts[(size_t)k].n_chunks;
                q.forward = k > 0;
                q.lam = pairs + (size_t)(at - 1) * 2 * E;
                q.rho = q.lam + E;
            }
            CK(cudaMemcpyAsync(c->gparts.p, c->gparts_host.data(), (size_t)K * sizeof(AdjPart),
                               cudaMemcpyHostToDevice, c->st));
        }
    }
    if (!c->grad.encoded) RC(encode_plan(c, c->grad));
    CK(cudaEventRecord(c->ev_ready, c->st));
    return STAB_OK;
}

}  // namespace

cudaStream_t stab::ctx_stream(stab_ctx *c) { return c ? c->st : nullptr; }
void stab::ctx_forget_sweep(stab_ctx *c) {
    if (c) c->tx_gen = -1;
}

extern "C" {

void stab_default_opts(stab_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->device = -1;
    o->kernel = STAB_KERNEL_AUTO;
    o->fuse = 1;
}

int stab_version(void) { return STAB_VERSION; }

namespace {

// What a kernel applies from a stream, in order: every pull record (last
// listed first), then, for a pass with ops, its header (pull count cleared)
// and its op records.  False when the stream is malformed (a record that is
// not a header where one is due, a pass straddling a chunk, no R_END) or its
// encoded positions are not those of its R_ROT / R_MAP3 records.
bool stream_actions(const std::vector<Rec> &s, const std::vector<int32_t> &enc,
                    std::vector<Rec> *out) {
    std::vector<int32_t> pos;
    size_t r = 0;
    while (r < s.size()) {
        const Rec &h = s[r];
        if (h.kind == R_END) return pos == enc;
        if (h.kind == R_NEXT) {
            r = (r / kChunkRecs + 1) * kChunkRecs;
            continue;
        }
        const size_t len = 1 + (size_t)h.param + (size_t)h.gate;
        if (h.kind != R_PASS || h.param < 0 || h.gate < 0 ||
            r / kChunkRecs != (r + len - 1) / kChunkRecs || r + len > s.size())
            return false;
        for (int k = h.param; k > 0; --k) out->push_back(s[r + (size_t)k]);
        if (h.gate > 0) {
            Rec hh = h;
            hh.param = 0;
            hh.code = 0;   // the repeated-pull hint is not an action
            out->push_back(hh);
            for (int k = 0; k < h.gate; ++k) {
                const size_t i = r + 1 + (size_t)h.param + (size_t)k;
                if (s[i].kind == R_ROT || s[i].kind == R_MAP3) pos.push_back((int32_t)i);
                out->push_back(s[i]);
            }
        }
        r += len;
    }
    return false;
}

// Every pass header of a one-piece stream carries kPullRepeat exactly when
// its pull records equal those of the previous pull pass.
bool pull_repeat_flags_exact(const std::vector<Rec> &s) {
    std::vector<Rec> last;
    size_t r = 0;
    while (r < s.size()) {
        const Rec &h = s[r];
        if (h.kind == R_END) return true;
        if (h.kind == R_NEXT) {
            r = (r / kChunkRecs + 1) * kChunkRecs;
            continue;
        }
        if (h.kind != R_PASS || h.param < 0 || h.gate < 0) return false;
        if (h.param > 0) {
            bool same = (size_t)h.param == last.size();
            for (int k = 0; same && k < h.param; ++k) {
                const Rec &p = s[r + 1 + (size_t)k];
                same = p.kind == last[(size_t)k].kind && p.q == last[(size_t)k].q &&
                       p.q1 == last[(size_t)k].q1;
            }
            if (same != (h.code == kPullRepeat)) return false;
            last.assign(s.begin() + (long)r + 1, s.begin() + (long)r + 1 + h.param);
        } else if (h.code != 0) {
            return false;
        }
        r += 1 + (size_t)h.param + (size_t)h.gate;
    }
    return false;
}

}  // namespace

int stab_selftest_plan(int n, const stab_gate *gates, int64_t m, int64_t n_params, int mode) {
    if (n < 1 || n > STAB_MAX_QUBITS) return STAB_E_RANGE;
    if (mode < 0 || mode > 3) return STAB_E_RANGE;
    std::string msg;
    RC(validate_gates(n, gates, m, n_params, &msg));
    const PlanMode pm = mode == 0 ? PLAN_FUSED : mode == 1 ? PLAN_GRAD : mode == 2 ? PLAN_PLAIN
                                                                               : PLAN_ROWS;
    HostPlan a, b;
    build_plan(n, gates, m, n_params, pm, &a, false, true);
    build_plan(n, gates, m, n_params, pm, &b, false, false);
    auto same = [](const auto &x, const auto &y) {
        return x.size() == y.size() &&
               (x.empty() || std::memcmp(x.data(), y.data(), x.size() * sizeof(x[0])) == 0);
    };
    bool ok = same(a.passes, b.passes) && same(a.ops, b.ops) && same(a.maps, b.maps) &&
              same(a.map_gate_idx, b.map_gate_idx) && same(a.raw, b.raw) &&
              same(a.param_ptr, b.param_ptr) && same(a.param_rot, b.param_rot) &&
              a.n_rot == b.n_rot;
    for (bool backward : {false, true}) {
        std::vector<Rec> sa, sb;
        build_stream(a, backward, &sa);
        build_stream(b, backward, &sb);
        ok = ok && same(sa, sb) && pull_repeat_flags_exact(sa);
    }
    // one-piece against two-piece streams, compared as what a kernel applies:
    // pulls in application order, passes with ops (identity passes only pull)
    DevPlan P;
    P.host = std::move(b);
    const int np = (int)P.host.passes.size();
    for (bool backward : {false, true}) {
        DevStreamBuf one, two;
        build_streams(P, {{&one, backward, 0, np}}, false);
        build_streams(P, {{&two, backward, 0, np}}, true);
        std::vector<Rec> joined = two.host;
        joined.insert(joined.end(), two.tail.begin(), two.tail.end());
        std::vector<int32_t> enc = two.enc;
        enc.insert(enc.end(), two.tail_enc.begin(), two.tail_enc.end());
        std::vector<Rec> fa, fb;
        ok = ok && two.host.size() % kChunkRecs == 0 &&
             (size_t)two.n_chunks * kChunkRecs == joined.size() &&
             stream_actions(one.host, one.enc, &fa) && stream_actions(joined, enc, &fb) &&
             same(fa, fb);
    }
    return ok ? STAB_OK : STAB_E_STATE;
}

namespace {

// Rotation ordinals (sorted) and two-qubit gate count of passes [0, k) of a
// plan: maps list their gates, rotation ops carry their ordinals.
void prefix_content(const HostPlan &P, int k, std::vector<int32_t> *rots, int64_t *two_q) {
    rots->clear();
    *two_q = 0;
    for (int i = 0; i < k; ++i) {
        const DevPass &p = P.passes[(size_t)i];
        for (int j = 0; j < p.n_ops; ++j) {
            const DevOp &op = P.ops[p.first + (uint32_t)j];
            if (p.type == P_CLIFF) {
                ++*two_q;
            } else if (op.kind == K_ROT) {
                rots->push_back(op.gate);
            } else if (op.kind == K_MAP3) {
                const DevMap3 &mp = P.maps[(size_t)op.param];
                for (int g = 0; g < mp.count; ++g) {
                    const int32_t o = P.rot_ordinal[(size_t)P.map_gate_idx[(size_t)(mp.first + g)]];
                    if (o >= 0) rots->push_back(o);
                }
            }
        }
    }
    std::sort(rots->begin(), rots->end());
}

}  // namespace

int stab_selftest_align(int n, const stab_gate *gates, int64_t m, int64_t n_params,
                        int64_t *aligned) {
    if (n < 1 || n > STAB_MAX_QUBITS) return STAB_E_RANGE;
    std::string msg;
    RC(validate_gates(n, gates, m, n_params, &msg));
    HostPlan F, G;
    build_plan(n, gates, m, n_params, PLAN_ROWS, &F, false, true);
    build_plan(n, gates, m, n_params, PLAN_GRAD, &G, false, true);
    // rotation ordinals of the generator plan's maps need the gate -> ordinal table
    if (F.rot_ordinal.size() != (size_t)m) {
        F.rot_ordinal.assign((size_t)m, -1);
        int32_t nr = 0;
        for (int64_t i = 0; i < m; ++i)
            if (gates[i].op >= STAB_RX) F.rot_ordinal[(size_t)i] = nr++;
    }
    int64_t count = 0;
    bool refused = false;
    std::vector<int32_t> ra, rb;
    int64_t qa = 0, qb = 0;
    for (int k = 1; k < (int)F.passes.size(); ++k) {
        if (!unit_start(F, (size_t)k)) continue;
        const int g = aligned_pass(F, k, G);
        if (g < 0) {
            refused = true;
            break;
        }
        prefix_content(F, k, &ra, &qa);
        prefix_content(G, g, &rb, &qb);
        if (ra != rb || qa != qb) return STAB_E_STATE;
        ++count;
    }
    if (refused) {
        // the aligner refuses only where the plans' unit sequences differ
        std::vector<uint16_t> ua, ub;
        for (size_t i = 0; i < F.passes.size(); ++i)
            if (unit_start(F, i)) ua.push_back((uint16_t)(F.passes[i].type << 8 | F.passes[i].q));
        for (size_t i = 0; i < G.passes.size(); ++i)
            if (unit_start(G, i)) ub.push_back((uint16_t)(G.passes[i].type << 8 | G.passes[i].q));
        if (ua == ub) return STAB_E_STATE;
        count = 0;
    }
    if (aligned) *aligned = count;
    return STAB_OK;
}

int stab_selftest_bounded_wait(int64_t polls) {
    if (polls < 0) return STAB_E_RANGE;
    cudaStream_t s = nullptr;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    int32_t *d = nullptr;
    int32_t h = -1;
    cudaError_t e = cudaMallocAsync(&d, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_bounded_wait(polls, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (d) cudaFreeAsync(d, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (e == cudaSuccess) e = e2;
    CK(e);
    return h == 0 ? STAB_OK : STAB_E_TIMEOUT;
}

int stab_last_cuda_error(void) { return g_last_cuda; }

const char *stab_error_string(int s) {
    switch (s) {
    case STAB_OK: return "ok";
    case STAB_E_INVAL: return "invalid argument";
    case STAB_E_RANGE: return "value out of range";
    case STAB_E_NOMEM: return "out of device memory";
    case STAB_E_TIMEOUT: return "device wait timed out";
    case STAB_E_NONFINITE: return "non-finite angle or coefficient";
    case STAB_E_CUDA: return "CUDA runtime error";
    case STAB_E_STATE: return "call out of order";
    case STAB_E_BUSY: return "queue full";
    default: return "unknown status";
    }
}

namespace {

int create_ctx(int n, const stab_opts *opts, const stab_path_choice *forced, stab_ctx **out) {
    if (!out) return STAB_E_INVAL;
    *out = nullptr;
    if (n < 1 || n > STAB_MAX_QUBITS) return STAB_E_RANGE;
    stab_opts o;
    stab_default_opts(&o);
    if (opts) o = *opts;
    if (o.kernel < STAB_KERNEL_AUTO || o.kernel > STAB_KERNEL_PLAIN) return STAB_E_INVAL;
    if (o.kernel == STAB_KERNEL_RESIDENT && n > kMaxResidentQubits) return STAB_E_RANGE;
    if ((o.alloc == nullptr) != (o.free == nullptr)) return STAB_E_INVAL;
    int dev = o.device;
    cudaError_t e = cudaSuccess;
    if (dev < 0) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        return STAB_E_CUDA;
    }
    // the path the context runs: the tuner's choice for AUTO (measured on
    // first use of this n on this GPU model), the defaults otherwise
    stab_path_choice choice;
    stab_path_defaults(n, &choice);
    if (forced) choice = *forced;
    else if (o.kernel == STAB_KERNEL_AUTO && o.fuse) RC(resolve_path_choice(dev, n, &o, &choice));
    stab_ctx *c = new (std::nothrow) stab_ctx();
    if (!c) return STAB_E_NOMEM;
    c->n = n;
    c->fwd.host_n = c->grad.host_n = n;
    c->kernel = o.kernel;
    c->fuse = o.fuse;
    c->choice = choice;
    c->alloc = o.alloc;
    c->free = o.free;
    c->user = o.alloc_user;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        c->device = dev;
        if (o.stream || o.stream_given) {
            c->st = (cudaStream_t)o.stream;
        } else {
            e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
            c->own_st = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_tx, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_aux, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_stage, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_stage, c->st);
    if (e == cudaSuccess) {
        const int r = c->dalloc(c->status, 256, c->st);
        if (r != STAB_OK) {
            stab_destroy(c);
            return r;
        }
        e = cudaMemsetAsync(c->status.p, 0, 256, c->st);
    }
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        stab_destroy(c);
        return STAB_E_CUDA;
    }
    *out = c;
    return STAB_OK;
}

}  // namespace

}  // extern "C"

int stab::create_with_choice(int n, const stab_opts *opts, const stab_path_choice *choice,
                             stab_ctx **out) {
    if (!choice) return STAB_E_INVAL;
    return create_ctx(n, opts, choice, out);
}

extern "C" {

int stab_create(int n, const stab_opts *opts, stab_ctx **out) {
    return create_ctx(n, opts, nullptr, out);
}

int stab_path_current(stab_ctx *c, stab_path_choice *out) {
    if (!c || !out) return STAB_E_INVAL;
    *out = c->choice;
    return STAB_OK;
}

int stab_destroy(stab_ctx *c) {
    if (!c) return STAB_OK;
    cudaSetDevice(c->device);
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->aux) cudaStreamSynchronize(c->aux);
    if (c->aux2) cudaStreamSynchronize(c->aux2);
    c->g_gens.reset();
    c->g_expect.reset();
    c->g_grad.reset();
    DevBuf *bufs[] = {&c->fwd.buf, &c->grad.buf, &c->thetas, &c->gens, &c->gens_tmp, &c->lam,
                      &c->rho, &c->tmp, &c->tmp2, &c->terms, &c->scal, &c->grad_rot,
                      &c->partials, &c->grads, &c->status, &c->gbuf, &c->lam2, &c->tmp3,
                      &c->dotbuf, &c->tmat, &c->avec, &c->rmid, &c->lmid, &c->bterms,
                      &c->units_g, &c->units_e, &c->cnt, &c->gmid, &c->chainbuf,
                      &c->chainbuf_e, &c->odense, &c->gpairs, &c->gparts};
    for (DevBuf *b : bufs) c->dfree(*b, c->st);
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->stage) cudaFreeHost(c->stage);
    if (c->aux_stage) cudaFreeHost(c->aux_stage);
    if (c->ev_ready) cudaEventDestroy(c->ev_ready);
    if (c->ev_tx) cudaEventDestroy(c->ev_tx);
    if (c->ev_aux) cudaEventDestroy(c->ev_aux);
    if (c->ev_stage) cudaEventDestroy(c->ev_stage);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->aux2) cudaStreamDestroy(c->aux2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_st && c->st) cudaStreamDestroy(c->st);
    delete c;
    return STAB_OK;
}

int stab_load_circuit(stab_ctx *c, const stab_gate *gates, int64_t m, const double *thetas,
                      int64_t n_params) {
    if (!c) return STAB_E_INVAL;
    std::string msg;
    RC(validate_gates(c->n, gates, m, n_params, &msg));
    RC(validate_thetas(thetas, n_params));
    CK(cudaSetDevice(c->device));
    // new state is built before the old one is dropped only where cheap; on an
    // error below the context reports STAB_E_STATE until a load succeeds
    c->loaded = false;
    c->gens_valid = false;
    c->gates.assign(gates, gates + m);
    c->n_params = n_params;
    c->grad.built = false;
    c->grad.encoded = false;
    reset_graphs(c);
    build_plan(c->n, gates, m, n_params, c->fwd_mode(), &c->fwd.host, !c->use_resident());
    if (c->use_resident()) {
        // split streams for the resident sweeps: generators through the
        // transfer matrix of the second part (n <= 4), expectations meeting in
        // the middle.  The cut balances the two parts' pass times; at n = 4,
        // where k_transfer_cols carries two columns per CTA at a different
        // pass rate than a first-part unit alone on its SM, the path tuner
        // times candidate cuts (n <= 3: every unit has an SM to itself, half).
        // At n = 4 the tuner may also cut the plan in three (a first part of
        // gen_cut of the passes, then two equal parts whose transfer matrices
        // share the SMs four columns to an SM).
        const bool split = c->kernel == STAB_KERNEL_AUTO && c->fuse;
        const double cut = c->choice.gen_cut;
        const int np = (int)c->fwd.host.passes.size();
        int parts = split ? chain_parts(c) : 2;
        double first = 0.0;
        if (split && transfer_cols_ctas(c->n) > 0 && c->choice.gen_parts == 3 &&
            np >= 3 * kSplitMinPasses) {
            parts = 3;
            first = cut;
        }
        make_streams(c->fwd, split ? cut : 0.0, false, parts, first);
    }
    else no_streams(c->fwd);
    RC(upload_thetas_host(c, thetas));
    RC(upload_plan(c, c->fwd));
    RC(encode_plan(c, c->fwd));
    CK(cudaEventRecord(c->ev_ready, c->st));
    c->param_gen++;
    c->loaded = true;
    return STAB_OK;
}

int stab_set_params(stab_ctx *c, const double *thetas, int is_device) {
    if (!c) return STAB_E_INVAL;
    if (!c->loaded) return STAB_E_STATE;
    CK(cudaSetDevice(c->device));
    if (is_device) {
        if (c->n_params > 0) {
            if (!thetas) return STAB_E_INVAL;
            CK(cudaMemcpyAsync(c->thetas.p, thetas, (size_t)c->n_params * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->st));
        }
    } else {
        RC(validate_thetas(thetas, c->n_params));
        RC(upload_thetas_host(c, thetas));
    }
    RC(encode_plan(c, c->fwd));
    c->grad.encoded = false;
    c->gens_valid = false;
    c->param_gen++;
    CK(cudaEventRecord(c->ev_ready, c->st));
    return STAB_OK;
}

int stab_run_generators(stab_ctx *c) {
    if (!c) return STAB_E_INVAL;
    if (!c->loaded) return STAB_E_STATE;
    CK(cudaSetDevice(c->device));
    const int n = c->n;
    const size_t bytes = c->vec_bytes() * (size_t)n;
    RC(c->dalloc(c->gens, bytes, c->st));
    if (c->use_resident() && split_gens_ok(c)) {
        // the split sweep for these angles may already have run (for <O> or
        // the density matrix); then only the products with T remain
        if (c->tx_gen != c->param_gen) RC(split_run_g(c));
        RC(split_apply(c, 0, n, (double *)c->gens.p, nullptr, 0, nullptr, c->st));
        c->gens_cur = (double *)c->gens.p;
    } else if (c->use_resident()) {
        StreamArgs a{};
        a.stream = c->fwd.sf.dev;
        a.n_chunks = c->fwd.sf.n_chunks;
        a.init = INIT_GENERATOR;
        a.n_vec = n;
        a.out = (double *)c->gens.p;
        a.status = (int32_t *)c->status.p;
        CK(launch_resident_stream(n, a, c->st));
        c->launches++;
        c->gens_cur = (double *)c->gens.p;
    } else {
        RC(c->dalloc(c->gens_tmp, bytes, c->st));
        cudaStream_t s = c->aux;
        CK(cudaStreamWaitEvent(s, c->ev_ready, 0));
        const std::vector<const void *> key = {(const void *)c->plan_gen, c->gens.p,
                                               c->gens_tmp.p};
        RC(run_graph(c, c->g_gens, key, s, [&](cudaStream_t gs, void **result) {
            double *cur = (double *)c->gens.p, *alt = (double *)c->gens_tmp.p;
            CK(launch_fill(cur, n, n, INIT_GENERATOR, nullptr, 0, gs));
            c->launches++;
            RC(run_streamed(c, c->fwd, &cur, &alt, n, 0, gs));
            *result = cur;
            return STAB_OK;
        }));
        c->gens_cur = (double *)c->g_gens.result;
        CK(cudaEventRecord(c->ev_aux, s));
        CK(cudaStreamWaitEvent(c->st, c->ev_aux, 0));
    }
    c->gens_valid = true;
    return STAB_OK;
}

int stab_apply_circuit(stab_ctx *c, const stab_gate *gates, int64_t m, const double *thetas,
                       int64_t n_params) {
    RC(stab_load_circuit(c, gates, m, thetas, n_params));
    return stab_run_generators(c);
}

int stab_get_generators(stab_ctx *c, double *out, int out_is_device) {
    if (!c || !out) return STAB_E_INVAL;
    if (!c->gens_valid) return STAB_E_STATE;
    CK(cudaSetDevice(c->device));
    const size_t bytes = c->vec_bytes() * (size_t)c->n;
    if (out_is_device) {
        CK(cudaMemcpyAsync(out, c->gens_cur, bytes, cudaMemcpyDeviceToDevice, c->st));
    } else {
        CK(cudaMemcpyAsync(out, c->gens_cur, bytes, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        c->d2h_bytes += (int64_t)bytes;
        RC(check_status(c));
    }
    return STAB_OK;
}

const double *stab_generators_device(stab_ctx *c) {
    if (!c || !c->gens_valid) return nullptr;
    return c->gens_cur;
}

int stab_set_observable(stab_ctx *c, const stab_term *O, int64_t n_terms) {
    if (!c) return STAB_E_INVAL;
    CK(cudaSetDevice(c->device));
    c->obs_loaded = false;
    RC(upload_terms(c, O, n_terms));
    c->obs_loaded = true;
    return STAB_OK;
}

int stab_expect_async(stab_ctx *c, double *out_dev) {
    if (!c || !out_dev) return STAB_E_INVAL;
    if (!c->loaded || !c->obs_loaded) return STAB_E_STATE;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = c->aux;
    CK(cudaStreamWaitEvent(s, c->ev_ready, 0));
    const int32_t nt = c->n_obs_terms;
    if (c->use_resident() && chain_mode(c)) {
        // <O> = sum_P o_P r_P with r = T_K ... T_2 r_1 (Schroedinger picture;
        // the orthogonal maps make it equal to the x-free sum of U^dagger O U):
        // the generators' launch made for these angles carries rho_0 and the
        // parts' transfer matrices; else it runs here first
        if (c->tx_gen != c->param_gen) RC(split_run_g(c));
        CK(cudaStreamWaitEvent(s, c->ev_tx, 0));
        RC(split_apply(c, c->n, 1, nullptr, (const DevTerm *)c->terms.p, nt, out_dev, s));
    } else if (c->use_resident() && split_expect_ok(c)) {
        RC(split_units_e(c, s));
        BatchArgs a{};
        a.units = (const BatchUnit *)c->units_e.p;
        a.n_units = 2;
        a.counter = (int32_t *)c->cnt.p + 16;
        a.status = (int32_t *)c->status.p;
        CK(cudaMemsetAsync((int32_t *)c->cnt.p + 16, 0, 4, s));
        CK(launch_batch(a, 2, c->split_smem, s));
        CK(launch_dot((const double *)c->lmid.p, (const double *)c->rmid.p, c->n,
                      (double *)c->dotbuf.p, out_dev, s));
        c->launches += 3;
    } else if (c->use_resident()) {
        StreamArgs a{};
        a.stream = c->fwd.sb.dev;
        a.n_chunks = c->fwd.sb.n_chunks;
        a.init = INIT_TERMS;
        a.terms = (const DevTerm *)c->terms.p;
        a.n_terms = nt;
        a.n_vec = 1;
        a.xfree_out = out_dev;
        a.status = (int32_t *)c->status.p;
        CK(launch_resident_stream(c->n, a, s));
        c->launches++;
    } else {
        const size_t vb = c->vec_bytes();
        RC(c->dalloc(c->lam, vb, s));
        RC(c->dalloc(c->tmp, vb, s));
        RC(c->dalloc(c->scal, 64 * sizeof(double), s));
        // small vectors (the tile regime): O backward through the second half
        // of the circuit and rho_0 forward through the first half, at once on
        // two streams; <O> = <lambda_mid, r_mid> (orthogonal maps keep inner
        // products), half the sequential depth
        const bool split = c->fwd.host.mode != PLAN_PLAIN && c->fwd.host.mode != PLAN_PLAIN_ROWS &&
                           c->fwd.host.passes.size() >= 8;
        if (split) {
            RC(c->dalloc(c->lam2, vb, s));
            RC(c->dalloc(c->tmp3, vb, s));
            RC(c->dalloc(c->dotbuf, 256 * sizeof(double), s));
        }
        double *res = (double *)c->scal.p + 2;
        const std::vector<const void *> key = {(const void *)c->plan_gen, c->lam.p, c->tmp.p,
                                               c->lam2.p, c->tmp3.p, c->dotbuf.p,
                                               c->terms.p, (const void *)(intptr_t)nt, res,
                                               (const void *)(intptr_t)split};
        RC(run_graph(c, c->g_expect, key, s, [&](cudaStream_t gs, void **) {
            double *cur = (double *)c->lam.p, *alt = (double *)c->tmp.p;
            if (!split) {
                CK(launch_fill(cur, c->n, 1, INIT_TERMS, (const DevTerm *)c->terms.p, nt, gs));
                c->launches += nt ? 2 : 1;
                RC(run_streamed(c, c->fwd, &cur, &alt, 1, 1, gs));
                CK(launch_xfree_sum(cur, c->n, 1, res, gs));
                c->launches++;
                return STAB_OK;
            }
            const int np = (int)c->fwd.host.passes.size(), mid = np / 2;
            CK(cudaEventRecord(c->ev_fork, gs));
            CK(cudaStreamWaitEvent(c->aux2, c->ev_fork, 0));
            CK(launch_fill(cur, c->n, 1, INIT_TERMS, (const DevTerm *)c->terms.p, nt, gs));
            RC(run_streamed(c, c->fwd, &cur, &alt, 1, 1, gs, mid, np));
            double *rc = (double *)c->lam2.p, *ra = (double *)c->tmp3.p;
            CK(launch_fill(rc, c->n, 1, INIT_RHO0, nullptr, 0, c->aux2));
            RC(run_streamed(c, c->fwd, &rc, &ra, 1, 0, c->aux2, 0, mid));
            CK(cudaEventRecord(c->ev_join, c->aux2));
            CK(cudaStreamWaitEvent(gs, c->ev_join, 0));
            CK(launch_dot(cur, rc, c->n, (double *)c->dotbuf.p, res, gs));
            c->launches += (nt ? 2 : 1) + 1 + 2;
            return STAB_OK;
        }));
        CK(cudaMemcpyAsync(out_dev, res, sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    // join: later work on the main stream sees the result
    CK(cudaEventRecord(c->ev_aux, s));
    CK(cudaStreamWaitEvent(c->st, c->ev_aux, 0));
    return STAB_OK;
}

int stab_expect(stab_ctx *c, const stab_term *O, int64_t n_terms, double *out) {
    if (!c || !out) return STAB_E_INVAL;
    if (!c->loaded) return STAB_E_STATE;
    RC(stab_set_observable(c, O, n_terms));
    RC(c->dalloc(c->scal, 64 * sizeof(double), c->st));
    RC(stab_expect_async(c, (double *)c->scal.p));
    CK(cudaEventSynchronize(c->ev_stage));
    RC(c->host_stage(c->stage, c->stage_bytes, 64 * sizeof(double)));
    double *h = (double *)c->stage;
    CK(cudaMemcpyAsync(h, c->scal.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->d2h_bytes += (int64_t)sizeof(double);
    *out = *h;
    RC(check_status(c));
    return STAB_OK;
}

int stab_grad_async(stab_ctx *c, double *expect_dev, double *grads_dev) {
    if (!c) return STAB_E_INVAL;
    if (!c->loaded || !c->obs_loaded) return STAB_E_STATE;
    if (c->n_params > 0 && !grads_dev) return STAB_E_INVAL;
    CK(cudaSetDevice(c->device));
    RC(ensure_grad_plan(c));
    cudaStream_t s = c->aux;
    CK(cudaStreamWaitEvent(s, c->ev_ready, 0));
    const int32_t nt = c->n_obs_terms;
    const int n = c->n;
    const int n_rot = c->grad.host.n_rot;
    RC(c->dalloc(c->scal, 64 * sizeof(double), s));
    RC(c->dalloc(c->grad_rot, (size_t)(n_rot ? n_rot : 1) * sizeof(double), s));
    double *e_out = expect_dev ? expect_dev : (double *)c->scal.p + 1;
    // the resident sweeps store each thread's dot share per rotation (no
    // reduction on the sweep's critical path; one fixed-order sum after it)
    // while the CTA has at most kPartialThreads threads and the shares fit
    // kPartialBytes; otherwise each pass reduces its dots over the CTA
    double *partials = nullptr;
    const int part_threads = resident_adjoint_threads(n);
    if (c->use_resident_adjoint()) {
        const size_t bytes = resident_partial_bytes(n, n_rot);
        if (bytes > 0) {
            RC(c->dalloc(c->partials, bytes, s));
            partials = (double *)c->partials.p;
        }
    }
    if (c->use_resident_adjoint() && c->grad_aligned) {
        // the gradient plan's parts end where the generators' split sweep cuts
        // the circuit, so the pair at every cut comes from that sweep: rho_0
        // through the first part is its first-part vector, rho at a later cut
        // the next parts' transfer matrices applied to it, and lambda at a cut
        // is O carried backward through the parts after it, T_k^T (the maps
        // being orthogonal) from the last part to the first; the sweep is
        // reused when it was made for these angles.  Then every part is swept
        // at once: the first backward from its end, the others forward.
        if (c->tx_gen != c->param_gen) RC(split_run_g(c));
        CK(cudaStreamWaitEvent(s, c->ev_tx, 0));
        const int K = (int)c->grad_cuts.size() - 1;
        const size_t E = (size_t)1 << (2 * n), EE = E * E;
        RC(c->dalloc(c->odense, E * sizeof(double), s));
        double *o = (double *)c->odense.p;
        CK(launch_fill(o, n, 1, INIT_TERMS, (const DevTerm *)c->terms.p, nt, s));
        const double *T = (const double *)c->tmat.p;
        const double *r1 = (const double *)c->avec.p + (size_t)n * E;
        double *pairs = (double *)c->gpairs.p;
        auto lam = [&](int k) { return pairs + (size_t)(k - 1) * 2 * E; };
        if (n == 4) {
            CK(cudaMemcpyAsync(lam(1) + E, r1, E * sizeof(double), cudaMemcpyDeviceToDevice, s));
            for (int k = 1; k + 1 <= K - 1; ++k)
                CK(launch_apply_transfer(T + (size_t)(k - 1) * EE, lam(k) + E, lam(k + 1) + E, 1,
                                         n, s));
            for (int k = K - 1; k >= 1; --k)
                CK(launch_apply_transfer_t(T + (size_t)(k - 1) * EE, k == K - 1 ? o : lam(k + 1),
                                           lam(k), n, s));
            c->launches += 1 + 2 * (K - 1) - 1;
        } else {
            CK(launch_adjoint_pairs(T, K, n, r1, o, pairs, s));
            c->launches += 2;
        }
        AdjointSplitArgs a{};
        a.phase = 1;
        a.parts = (const AdjPart *)c->gparts.p;
        a.n_parts = K;
        a.grad_rot = (double *)c->grad_rot.p;
        a.partials = partials;
        a.expect_out = e_out;
        a.status = (int32_t *)c->status.p;
        CK(launch_adjoint_split(n, a, s));
        c->launches++;
        if (partials) {
            CK(launch_reduce_partials(partials, n_rot, part_threads, (double *)c->grad_rot.p, s));
            c->launches++;
        }
        if (c->n_params > 0) {
            CK(launch_gather_grads((const double *)c->grad_rot.p, c->grad.param_ptr,
                                   c->grad.param_rot, (int)c->n_params, grads_dev, s));
            c->launches++;
        }
    } else if (c->use_resident_adjoint() && c->grad.split >= 0) {
        // meet in the middle: rho_0 forward through the first part and O
        // backward through the second, then the pair at the cut backward
        // through the first part and forward through the second
        const size_t E = (size_t)1 << (2 * n);
        RC(c->dalloc(c->gmid, 2 * E * sizeof(double), s));
        AdjointSplitArgs a{};
        a.stream[0] = c->grad.h1.dev;
        a.n_chunks[0] = c->grad.h1.n_chunks;
        a.stream[1] = c->grad.h2b.dev;
        a.n_chunks[1] = c->grad.h2b.n_chunks;
        a.phase = 0;
        a.terms = (const DevTerm *)c->terms.p;
        a.n_terms = nt;
        a.rmid = (double *)c->gmid.p;
        a.lmid = (double *)c->gmid.p + E;
        a.grad_rot = (double *)c->grad_rot.p;
        a.partials = partials;
        a.expect_out = e_out;
        a.status = (int32_t *)c->status.p;
        CK(launch_adjoint_split(n, a, s));
        a.stream[0] = c->grad.h1b.dev;
        a.n_chunks[0] = c->grad.h1b.n_chunks;
        a.stream[1] = c->grad.h2.dev;
        a.n_chunks[1] = c->grad.h2.n_chunks;
        a.phase = 1;
        CK(launch_adjoint_split(n, a, s));
        c->launches += 2;
        if (partials) {
            CK(launch_reduce_partials(partials, n_rot, part_threads, (double *)c->grad_rot.p, s));
            c->launches++;
        }
        if (c->n_params > 0) {
            CK(launch_gather_grads((const double *)c->grad_rot.p, c->grad.param_ptr,
                                   c->grad.param_rot, (int)c->n_params, grads_dev, s));
            c->launches++;
        }
    } else if (c->use_resident_adjoint()) {
        AdjointStreamArgs a{};
        a.fwd = c->grad.sf.dev;
        a.bwd = c->grad.sb.dev;
        a.n_fwd_chunks = c->grad.sf.n_chunks;
        a.n_bwd_chunks = c->grad.sb.n_chunks;
        a.terms = (const DevTerm *)c->terms.p;
        a.n_terms = nt;
        a.grad_rot = (double *)c->grad_rot.p;
        a.partials = partials;
        a.expect_out = e_out;
        a.status = (int32_t *)c->status.p;
        CK(launch_adjoint_stream(n, a, s));
        c->launches++;
        if (partials) {
            CK(launch_reduce_partials(partials, n_rot, part_threads, (double *)c->grad_rot.p, s));
            c->launches++;
        }
        if (c->n_params > 0) {
            CK(launch_gather_grads((const double *)c->grad_rot.p, c->grad.param_ptr,
                                   c->grad.param_rot, (int)c->n_params, grads_dev, s));
            c->launches++;
        }
    } else {
        // lambda and rho are one contiguous pair (lambda first), ping-ponged
        // with a second pair, so a Clifford gather moves both in one launch
        const size_t vb = c->vec_bytes();
        const uint64_t E = 1ull << (2 * n);
        RC(c->dalloc(c->lam, 2 * vb, s));
        RC(c->dalloc(c->tmp, 2 * vb, s));
        RC(c->dalloc(c->gbuf, (size_t)(c->n_params ? c->n_params : 1) * sizeof(double), s));
        const int nb = adjoint_stream_blocks(n);
        RC(c->dalloc(c->partials, (size_t)(n_rot ? n_rot : 1) * nb * sizeof(double), s));
        double *res = (double *)c->scal.p + 3;
        const bool tiles = n <= kAdjTileMaxN;
        RC(c->dalloc(c->lam2, 2 * vb, s));
        RC(c->dalloc(c->tmp3, 2 * vb, s));
        const std::vector<const void *> key = {
            (const void *)c->plan_gen, c->lam.p, c->tmp.p, c->lam2.p, c->tmp3.p, c->partials.p,
            c->grad_rot.p, c->gbuf.p, c->terms.p, (const void *)(intptr_t)nt, res};
        {
            // Split sweep.  The circuit's passes are cut in two halves at
            // `mid`.  Phase 1, two branches at once: r forward through the
            // first half, lambda backward through the second; both meet at
            // `mid`.  Phase 2, two branches at once: the pair (lambda, r)
            // backward through the first half and forward through the second
            // (every map is orthogonal, so lambda moves forward as r does),
            // each rotation's dot taken at its post-gate pair.  Half the
            // sequential depth of forward-then-reverse, and two chains of
            // launches share the GPU (measured faster at every n: 1.6x at
            // n = 8, 1.1-1.3x at n = 9..12).
            RC(run_graph(c, c->g_grad, key, s, [&](cudaStream_t gs, void **) {
                const auto &passes = c->grad.host.passes;
                const int np = (int)passes.size(), mid = np / 2;
                const DevOp *ops = c->grad.prog.ops;
                const auto &hops = c->grad.host.ops;
                double *A = (double *)c->lam.p, *B = (double *)c->tmp.p;
                double *Cb = (double *)c->lam2.p, *D = (double *)c->tmp3.p;
                auto fork = [&](cudaStream_t from, cudaStream_t to) -> int {
                    CK(cudaEventRecord(c->ev_fork, from));
                    CK(cudaStreamWaitEvent(to, c->ev_fork, 0));
                    return STAB_OK;
                };
                auto join = [&](cudaStream_t from, cudaStream_t to) -> int {
                    CK(cudaEventRecord(c->ev_join, from));
                    CK(cudaStreamWaitEvent(to, c->ev_join, 0));
                    return STAB_OK;
                };
                // the adjoint sweep of passes [k0, k1) on a pair, one way
                auto sweep = [&](double *&pr, double *&al, int k0, int k1, bool forward,
                                 cudaStream_t st) -> int {
                    std::vector<const DevPass *> group;
                    std::vector<int> wires;
                    const DevPass *pending = nullptr;
                    auto gather_now = [&]() -> int {
                        CK(launch_stream_cliff(pr, al, n, 2, *pending, ops, forward ? 0 : 1, st));
                        c->launches++;
                        std::swap(pr, al);
                        pending = nullptr;
                        return STAB_OK;
                    };
                    auto flush = [&]() -> int {
                        if (group.empty()) return STAB_OK;
                        if (!tiles) {
                            for (const DevPass *gp : group) {
                                CK(launch_adjoint_wire(pr, pr + E, n, *gp, ops,
                                                       (double *)c->partials.p, forward ? 1 : 0,
                                                       st));
                                c->launches++;
                            }
                            group.clear();
                            wires.clear();
                            return STAB_OK;
                        }
                        TileGroup tg;
                        make_tile_group(n, 1, group, forward ? 0 : 1, &tg, nb,
                                        std::min(kAdjTileBits, 2 * n));
                        for (size_t j = 0; j < group.size(); ++j) {
                            int nr = 0;
                            for (int k = 0; k < group[j]->n_ops; ++k)
                                nr += hops[(size_t)group[j]->first + k].kind == K_ROT;
                            tg.n_rot[j] = (uint8_t)nr;
                        }
                        double *dst = pr;
                        if (pending) {
                            tg.pull_n = pending->n_ops;
                            tg.pull_first = pending->first;
                            tg.pull_inverse = forward ? 0 : 1;
                            dst = al;
                        }
                        CK(launch_adjoint_tile(pr, dst, n, tg, ops, (double *)c->partials.p, st));
                        c->launches++;
                        if (pending) {
                            std::swap(pr, al);
                            pending = nullptr;
                        }
                        group.clear();
                        wires.clear();
                        return STAB_OK;
                    };
                    for (int t = 0; t < k1 - k0; ++t) {
                        const DevPass &p = passes[forward ? k0 + t : k1 - 1 - t];
                        if (p.type == P_WIRE) {
                            const bool known =
                                std::find(wires.begin(), wires.end(), (int)p.q) != wires.end();
                            if ((int)group.size() == kTileMaxPasses ||
                                (!known && (int)wires.size() == kTileWires))
                                RC(flush());
                            group.push_back(&p);
                            if (!known) wires.push_back(p.q);
                            continue;
                        }
                        RC(flush());
                        if (pending) RC(gather_now());
                        if (p.type == P_TAB) {
                            CK(launch_stream_tab(pr, al, n, 2,
                                                 c->grad.prog.tabs + 2 * p.first + (forward ? 0 : 1),
                                                 st));
                            c->launches++;
                            std::swap(pr, al);
                            continue;
                        }
                        pending = &p;
                        if (!tiles) RC(gather_now());
                    }
                    RC(flush());
                    if (pending) RC(gather_now());
                    return STAB_OK;
                };
                // phase 1
                RC(fork(gs, c->aux2));
                double *rho = A + E, *rho_alt = B + E;
                CK(launch_fill(rho, n, 1, INIT_RHO0, nullptr, 0, gs));
                RC(run_streamed(c, c->grad, &rho, &rho_alt, 1, 0, gs, 0, mid));
                double *lam = Cb, *lam_alt = D;
                CK(launch_fill(lam, n, 1, INIT_TERMS, (const DevTerm *)c->terms.p, nt, c->aux2));
                RC(run_streamed(c, c->grad, &lam, &lam_alt, 1, 1, c->aux2, mid, np));
                c->launches += nt ? 3 : 2;
                RC(join(c->aux2, gs));
                // the meeting pair, once in each branch's buffers
                double *X = rho - E, *Xalt = X == A ? B : A;
                double *Y = lam, *Yalt = Y == Cb ? D : Cb;
                CK(cudaMemcpyAsync(X, lam, vb, cudaMemcpyDeviceToDevice, gs));
                CK(cudaMemcpyAsync(Y + E, rho, vb, cudaMemcpyDeviceToDevice, gs));
                // phase 2
                RC(fork(gs, c->aux2));
                RC(sweep(X, Xalt, 0, mid, false, gs));
                RC(sweep(Y, Yalt, mid, np, true, c->aux2));
                RC(join(c->aux2, gs));
                CK(launch_reduce_partials((const double *)c->partials.p, n_rot, nb,
                                          (double *)c->grad_rot.p, gs));
                CK(launch_xfree_sum(X, n, 1, res, gs));   // <O> = <lambda_0, rho_0>
                c->launches += 2;
                if (c->n_params > 0) {
                    CK(launch_gather_grads((const double *)c->grad_rot.p, c->grad.param_ptr,
                                           c->grad.param_rot, (int)c->n_params,
                                           (double *)c->gbuf.p, gs));
                    c->launches++;
                }
                return STAB_OK;
            }));
        }
        CK(cudaMemcpyAsync(e_out, res, sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (c->n_params > 0)
            CK(cudaMemcpyAsync(grads_dev, c->gbuf.p, (size_t)c->n_params * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaEventRecord(c->ev_aux, s));
    CK(cudaStreamWaitEvent(c->st, c->ev_aux, 0));
    return STAB_OK;
}

int stab_grad(stab_ctx *c, const stab_term *O, int64_t n_terms, double *expect_out,
              double *grads_out) {
    if (!c) return STAB_E_INVAL;
    if (!c->loaded) return STAB_E_STATE;
    if (c->n_params > 0 && !grads_out) return STAB_E_INVAL;
    RC(stab_set_observable(c, O, n_terms));
    RC(c->dalloc(c->grads, (size_t)(c->n_params ? c->n_params : 1) * sizeof(double), c->st));
    RC(c->dalloc(c->scal, 64 * sizeof(double), c->st));
    RC(stab_grad_async(c, (double *)c->scal.p, (double *)c->grads.p));
    const size_t gbytes = (size_t)c->n_params * sizeof(double);
    CK(cudaEventSynchronize(c->ev_stage));
    RC(c->host_stage(c->stage, c->stage_bytes, gbytes + 64 * sizeof(double)));
    double *h = (double *)c->stage;
    CK(cudaMemcpyAsync(h, c->scal.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (gbytes) CK(cudaMemcpyAsync(h + 8, c->grads.p, gbytes, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->d2h_bytes += (int64_t)(gbytes + sizeof(double));
    if (expect_out) *expect_out = h[0];
    if (gbytes) std::memcpy(grads_out, h + 8, gbytes);
    RC(check_status(c));
    return STAB_OK;
}

int stab_density_matrix(stab_ctx *c, double *out, int out_is_device) {
    if (!c || !out) return STAB_E_INVAL;
    if (!c->loaded) return STAB_E_STATE;
    CK(cudaSetDevice(c->device));
    const int n = c->n;
    const size_t vb = c->vec_bytes();
    RC(c->dalloc(c->rho, vb, c->st));
    double *r = (double *)c->rho.p;
    if (c->use_resident() && split_gens_ok(c)) {
        // r = T r_1: rho_0 through the first part, then the later parts'
        // transfer matrices (built alongside, as for the generators; reused
        // when the sweep for these angles has run)
        if (c->tx_gen != c->param_gen) RC(split_run_g(c));
        RC(split_apply(c, n, 1, r, nullptr, 0, nullptr, c->st));
    } else if (c->use_resident()) {
        StreamArgs a{};
        a.stream = c->fwd.sf.dev;
        a.n_chunks = c->fwd.sf.n_chunks;
        a.init = INIT_RHO0;
        a.n_vec = 1;
        a.out = r;
        a.status = (int32_t *)c->status.p;
        CK(launch_resident_stream(n, a, c->st));
        c->launches++;
    } else {
        RC(c->dalloc(c->tmp2, vb, c->st));
        double *cur = r, *alt = (double *)c->tmp2.p;
        CK(launch_fill(cur, n, 1, INIT_RHO0, nullptr, 0, c->st));
        c->launches++;
        RC(run_streamed(c, c->fwd, &cur, &alt, 1, 0, c->st));
        r = cur;
    }
    const size_t rho_bytes = 2 * vb;
    if (out_is_device) {
        CK(launch_decode_rho(r, n, out, c->st));
        c->launches++;
        return STAB_OK;
    }
    RC(c->dalloc(c->tmp, rho_bytes, c->st));
    CK(launch_decode_rho(r, n, (double *)c->tmp.p, c->st));
    c->launches++;
    CK(cudaMemcpyAsync(out, c->tmp.p, rho_bytes, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->d2h_bytes += (int64_t)rho_bytes;
    return check_status(c);
}

int stab_synchronize(stab_ctx *c) {
    if (!c) return STAB_E_INVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->st));
    CK(cudaStreamSynchronize(c->aux));
    return check_status(c);
}

int stab_plan_info(stab_ctx *c, int64_t *n_gates, int64_t *n_passes, int32_t *kernel) {
    if (!c) return STAB_E_INVAL;
    if (n_gates) *n_gates = (int64_t)c->gates.size();
    if (n_passes) *n_passes = (int64_t)c->fwd.host.passes.size();
    if (kernel) *kernel = c->use_resident() ? STAB_KERNEL_RESIDENT : STAB_KERNEL_STREAMED;
    return STAB_OK;
}

int stab_split_info(stab_ctx *c, int64_t *cut, int32_t *gen_units, int32_t *expect_units) {
    if (!c) return STAB_E_INVAL;
    const bool on = c->loaded && c->use_resident() && c->fwd.split >= 0;
    const int E = 1 << (2 * c->n);
    if (cut) *cut = on ? c->fwd.split : -1;
    const int n_mats = chain_mode(c) ? (int)c->fwd.parts.size() - 1 : 1;
    if (gen_units) *gen_units = on && split_gens_ok(c) ? c->n + 1 + n_mats * (E - 1) : 0;
    if (expect_units) *expect_units = on && !chain_mode(c) && split_expect_ok(c) ? 2 : 0;
    return STAB_OK;
}

int64_t stab_launch_count(stab_ctx *c) { return c ? c->launches : 0; }

int stab_grad_parts(stab_ctx *c, int32_t *parts) {
    if (!c || !parts) return STAB_E_INVAL;
    *parts = !c->grad.built ? 0 : c->grad_aligned ? (int32_t)c->grad_cuts.size() - 1 : 1;
    return STAB_OK;
}

int stab_transfer_bytes(stab_ctx *c, int64_t *h2d, int64_t *d2h) {
    if (!c) return STAB_E_INVAL;
    if (h2d) *h2d = c->h2d_bytes;
    if (d2h) *d2h = c->d2h_bytes;
    return STAB_OK;
}

}  // extern "C"

// Expectation of an observable already on the device as deduplicated terms
// (the sparse path's list when it switches to the dense vector).
int stab::expect_device_terms(stab_ctx *c, const DevTerm *terms, int64_t nt, double *out) {
    if (!c || !out || nt < 0 || nt > INT32_MAX || (nt > 0 && !terms)) return STAB_E_INVAL;
    if (!c->loaded) return STAB_E_STATE;
    CK(cudaSetDevice(c->device));
    c->obs_loaded = false;
    CK(cudaStreamSynchronize(c->aux));
    RC(c->dalloc(c->terms, (size_t)(nt ? nt : 1) * sizeof(DevTerm), c->st));
    if (nt)
        CK(cudaMemcpyAsync(c->terms.p, terms, (size_t)nt * sizeof(DevTerm),
                           cudaMemcpyDeviceToDevice, c->st));
    c->n_obs_terms = (int32_t)nt;
    CK(cudaEventRecord(c->ev_ready, c->st));
    c->obs_loaded = true;
    RC(c->dalloc(c->scal, 64 * sizeof(double), c->st));
    RC(stab_expect_async(c, (double *)c->scal.p));
    CK(cudaEventSynchronize(c->ev_stage));
    RC(c->host_stage(c->stage, c->stage_bytes, 64 * sizeof(double)));
    double *h = (double *)c->stage;
    CK(cudaMemcpyAsync(h, c->scal.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->d2h_bytes += (int64_t)sizeof(double);
    *out = *h;
    RC(check_status(c));
    return STAB_OK;
}

