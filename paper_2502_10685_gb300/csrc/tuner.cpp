// tuner.cpp -- stab_path_*: the choices of the single-circuit path (which
// kernels a STAB_KERNEL_AUTO context uses for n qubits), measured per GPU
// model and kept in a process-wide cache.
//
// The choices are the ones a fixed threshold would otherwise make: whether
// n = 5, 6 vectors stay resident in shared memory (one CTA each) or stream
// through HBM, for <O> and for gradients; where the generators' split sweep
// cuts the plan at n = 4 (the first part's vectors and the second part's
// transfer-matrix columns run on different kernels at different speeds, and
// the cut that makes them end together depends on both); and up to which
// launch size consecutive wire passes of a streamed plan share one
// tile-fused launch.  Each is timed on a probe circuit, candidate against
// candidate, through the public entry points of contexts created with the
// candidate's choice.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/stab.h"
#include "launch.h"
#include "tuner.h"

namespace stab {

namespace {

std::mutex g_mu;        // the cache
std::map<std::pair<std::string, int>, stab_path_choice> g_cache;
bool g_file_read = false;
std::mutex g_tune_mu;   // one tuning at a time (it creates contexts of its own)

bool name_ok(const char *name) {
    if (!name || !name[0]) return false;
    const size_t len = std::strlen(name);
    if (len > 255) return false;
    for (size_t i = 0; i < len; ++i)
        if (name[i] == '\t' || name[i] == '\n' || name[i] == '\r') return false;
    return true;
}

bool choice_ok(const stab_path_choice &c) {
    return (c.resident == 0 || c.resident == 1) &&
           (c.resident_adjoint == 0 || c.resident_adjoint == 1) && std::isfinite(c.gen_cut) &&
           c.gen_cut >= 0.3 && c.gen_cut <= 0.7 && c.tile_limit >= 0 &&
           (c.tuned == 0 || c.tuned == 1) && (c.gen_parts == 2 || c.gen_parts == 3);
}

const char *cache_file() {
    const char *p = std::getenv("STAB_PATH_CACHE");
    return (p && p[0]) ? p : nullptr;
}

bool tuning_enabled() {
    const char *v = std::getenv("STAB_PATH_TUNE");
    return !(v && std::strcmp(v, "0") == 0);
}

// Parses the cache file into `out`; false on any malformed line.
bool read_file(const char *path, std::map<std::pair<std::string, int>, stab_path_choice> *out,
               bool *opened) {
    *opened = false;
    FILE *f = std::fopen(path, "r");
    if (!f) return true;
    *opened = true;
    char line[512];
    bool ok = true;
    while (ok && std::fgets(line, sizeof line, f)) {
        size_t len = std::strlen(line);
        if (len == sizeof line - 1 && line[len - 1] != '\n') {
            ok = false;
            break;
        }
        while (len && (line[len - 1] == '\n' || line[len - 1] == '\r')) line[--len] = 0;
        if (!len) continue;
        char *tab = std::strchr(line, '\t');
        if (!tab) {
            ok = false;
            break;
        }
        *tab = 0;
        stab_path_choice c{};
        int n = 0, res = 0, radj = 0, tuned = 0, parts = 0;
        long long tl = 0;
        double cut = 0.0;
        char tail = 0;
        if (std::sscanf(tab + 1, "%d\t%d\t%d\t%lf\t%lld\t%d\t%d%c", &n, &res, &radj, &cut, &tl,
                        &tuned, &parts, &tail) != 7) {
            ok = false;
            break;
        }
        c.resident = res;
        c.resident_adjoint = radj;
        c.gen_cut = cut;
        c.tile_limit = tl;
        c.tuned = tuned;
        c.gen_parts = parts;
        if (!name_ok(line) || n < 1 || n > STAB_MAX_QUBITS || !choice_ok(c)) {
            ok = false;
            break;
        }
        (*out)[{std::string(line), n}] = c;
    }
    std::fclose(f);
    return ok;
}

bool write_file(const char *path) {
    FILE *f = std::fopen(path, "w");
    if (!f) return false;
    for (const auto &kv : g_cache) {
        const stab_path_choice &c = kv.second;
        std::fprintf(f, "%s\t%d\t%d\t%d\t%.17g\t%lld\t%d\t%d\n", kv.first.first.c_str(),
                     kv.first.second, c.resident, c.resident_adjoint, c.gen_cut,
                     (long long)c.tile_limit, c.tuned, c.gen_parts);
    }
    return std::fclose(f) == 0;
}

// First lookup: the file named by STAB_PATH_CACHE (caller holds g_mu).
void read_env_file_locked() {
    if (g_file_read) return;
    g_file_read = true;
    const char *p = cache_file();
    if (!p) return;
    std::map<std::pair<std::string, int>, stab_path_choice> m;
    bool opened = false;
    if (read_file(p, &m, &opened))
        for (auto &kv : m) g_cache[kv.first] = kv.second;
}

int device_name(int device, std::string *out) {
    cudaDeviceProp p;
    cudaError_t e = cudaGetDeviceProperties(&p, device);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return STAB_E_CUDA;
    }
    p.name[sizeof p.name - 1] = 0;
    *out = p.name;
    for (char &ch : *out)
        if (ch == '\t' || ch == '\n' || ch == '\r') ch = ' ';
    return STAB_OK;
}

// ---------------------------------------------------------------- probes

// The probe: a layered ansatz (R_x, R_y, R_z on every qubit, then the CNOT
// ring q -> q + 1 mod n), m gates, one angle slot per rotation, angles from a
// fixed 64-bit LCG spread over [0, 2 pi).
void probe_circuit(int n, int m, std::vector<stab_gate> *g, std::vector<double> *th) {
    g->clear();
    th->clear();
    uint64_t x = 0x9e3779b97f4a7c15ull;
    while ((int)g->size() < m) {
        for (int q = 0; q < n && (int)g->size() < m; ++q) {
            for (int op : {STAB_RX, STAB_RY, STAB_RZ}) {
                if ((int)g->size() >= m) break;
                x = x * 6364136223846793005ull + 1442695040888963407ull;
                th->push_back((double)(x >> 11) * (6.283185307179586 / 9007199254740992.0));
                g->push_back({(uint8_t)op, (uint8_t)q, 0, 0, (int32_t)th->size() - 1});
            }
        }
        if (n >= 2)
            for (int q = 0; q < n && (int)g->size() < m; ++q)
                g->push_back({(uint8_t)STAB_CX, (uint8_t)q, (uint8_t)((q + 1) % n), 0, -1});
    }
}

std::vector<stab_term> probe_observable(int n) {
    std::vector<stab_term> t;
    for (int q = 0; q + 1 < n; ++q) t.push_back({1.0, 0, (3ull << q)});
    for (int q = 0; q < n; ++q) t.push_back({0.5, 1ull << q, 0});
    return t;
}

enum ProbeOp { PR_GENS, PR_EXPECT, PR_GRAD };

struct Probe {
    int n, m;
    std::vector<stab_gate> g;
    std::vector<double> th;
    std::vector<stab_term> obs;
};

// Best device time (ms) of `op` on a context of the probe's size run with
// `choice`: two untimed calls (the second also captures the streamed
// sequences into their graphs), then the best of five timed ones.
int time_op(int device, const stab_opts *like, const Probe &P, const stab_path_choice &choice,
            ProbeOp op, float *best) {
    stab_opts o;
    stab_default_opts(&o);
    if (like) {
        // the creating context's allocator hooks; the probes run on streams
        // of their own, so nothing lands on the caller's stream (or in a
        // capture running on it), and every block is handed back after a
        // synchronize
        o.alloc = like->alloc;
        o.free = like->free;
        o.alloc_user = like->alloc_user;
    }
    o.device = device;
    stab_ctx *c = nullptr;
    int rc = create_with_choice(P.n, &o, &choice, &c);
    if (rc != STAB_OK) return rc;
    double *dev = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = ctx_stream(c);
    rc = stab_load_circuit(c, P.g.data(), (int64_t)P.g.size(), P.th.data(), (int64_t)P.th.size());
    if (rc == STAB_OK && op != PR_GENS)
        rc = stab_set_observable(c, P.obs.data(), (int64_t)P.obs.size());
    cudaError_t e = cudaSuccess;
    const size_t dev_bytes = (P.th.size() + 8) * sizeof(double);
    if (rc == STAB_OK) {
        if (o.alloc) {
            dev = (double *)o.alloc(dev_bytes, (void *)st, o.alloc_user);
            if (!dev) rc = STAB_E_NOMEM;
        } else {
            e = cudaMallocAsync((void **)&dev, dev_bytes, st);
        }
    }
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (rc == STAB_OK && e != cudaSuccess) {
        record_cuda_error(e);
        rc = STAB_E_CUDA;
    }
    auto call = [&]() {
        if (op == PR_GENS) {
            // every timed call runs the whole sweep (a repeated call for the
            // same angles would otherwise reuse the previous one)
            ctx_forget_sweep(c);
            return stab_run_generators(c);
        }
        if (op == PR_EXPECT) return stab_expect_async(c, dev);
        return stab_grad_async(c, dev, dev + 8);
    };
    float b = 1e30f;
    for (int k = 0; k < 7 && rc == STAB_OK; ++k) {
        if (k >= 2 && cudaEventRecord(e0, st) != cudaSuccess) rc = STAB_E_CUDA;
        if (rc == STAB_OK) rc = call();
        if (rc == STAB_OK && k >= 2) {
            float ms = 0.0f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = STAB_E_CUDA;
            else if (ms < b)
                b = ms;
        }
    }
    if (rc == STAB_OK) rc = stab_synchronize(c);
    cudaStreamSynchronize(st);
    if (dev) {
        if (o.free) o.free(dev, dev_bytes, (void *)st, o.alloc_user);
        else cudaFreeAsync(dev, st);
    }
    cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    stab_destroy(c);
    *best = b;
    return rc;
}

// A candidate replaces the default only when it is faster by more than this
// fraction: the probes' timings vary by about a percent from run to run, and
// a choice that flips with that noise would make the path vary between
// processes for no gain.
constexpr float kMargin = 0.02f;

bool clearly_faster(float t, float t_default) { return t < (1.0f - kMargin) * t_default; }

int measure(int device, const stab_opts *like, int n, stab_path_choice *out) {
    stab_path_choice d;
    stab_path_defaults(n, &d);
    d.tuned = 1;
    Probe P;
    P.n = n;
    if (n == 4) {
        // long enough (about 7,500 passes) that a pass's cost, not the
        // launch and staging overhead, decides between the cuts
        P.m = 24000;
        probe_circuit(n, P.m, &P.g, &P.th);
        const double def = d.gen_cut;
        float t_def = 0.0f, best = 1e30f;
        double best_cut = def;
        int best_parts = 2;
        struct Cand {
            int parts;
            double cut;
        };
        const Cand cands[] = {{2, 0.50}, {2, 0.53}, {2, 0.56}, {2, 0.59}, {2, 0.62},
                              {3, 0.43}, {3, 0.45}, {3, 0.47}, {3, 0.49}, {3, 0.51}};
        for (const Cand &k : cands) {
            stab_path_choice c = d;
            c.gen_cut = k.cut;
            c.gen_parts = k.parts;
            float t = 0.0f;
            int rc = time_op(device, like, P, c, PR_GENS, &t);
            if (rc != STAB_OK) return rc;
            if (k.parts == 2 && k.cut == def) t_def = t;
            if (t < best) {
                best = t;
                best_cut = k.cut;
                best_parts = k.parts;
            }
        }
        if (clearly_faster(best, t_def)) {
            d.gen_cut = best_cut;
            d.gen_parts = best_parts;
        }
    } else if (n == 5 || n == 6) {
        P.m = 2000;
        probe_circuit(n, P.m, &P.g, &P.th);
        P.obs = probe_observable(n);
        float t[2][2];   // [op: expect, grad][resident 0 / 1]
        for (int r = 0; r < 2; ++r) {
            stab_path_choice c = d;
            c.resident = c.resident_adjoint = r;
            int rc = time_op(device, like, P, c, PR_EXPECT, &t[0][r]);
            if (rc == STAB_OK) rc = time_op(device, like, P, c, PR_GRAD, &t[1][r]);
            if (rc != STAB_OK) return rc;
        }
        // the defaults are resident; streamed only when clearly faster
        d.resident = clearly_faster(t[0][0], t[0][1]) ? 0 : 1;
        d.resident_adjoint = clearly_faster(t[1][0], t[1][1]) ? 0 : 1;
    } else if (n >= 7 && n <= 9) {
        P.m = n == 7 ? 400 : (n == 8 ? 300 : 200);
        probe_circuit(n, P.m, &P.g, &P.th);
        P.obs = probe_observable(n);
        const int64_t E = (int64_t)1 << (2 * n);
        int64_t limit = 0;
        // one vector (<O>), then n vectors (the generators)
        for (ProbeOp op : {PR_EXPECT, PR_GENS}) {
            const int64_t size = E * (op == PR_GENS ? n : 1);
            stab_path_choice on = d, off = d;
            on.tile_limit = size;
            off.tile_limit = size - 1;
            float t_on = 0.0f, t_off = 0.0f;
            int rc = time_op(device, like, P, on, op, &t_on);
            if (rc == STAB_OK) rc = time_op(device, like, P, off, op, &t_off);
            if (rc != STAB_OK) return rc;
            // the default (tiles up to 2^17 entries) stands unless the other
            // form is clearly faster at this size
            const bool tiles_default = size <= d.tile_limit;
            const bool tiles = tiles_default ? !clearly_faster(t_off, t_on)
                                             : clearly_faster(t_on, t_off);
            if (tiles) limit = size;
        }
        d.tile_limit = limit;
    }
    *out = d;
    return STAB_OK;
}

// Measures and stores the choice (caller holds g_tune_mu).
int tune_locked(int device, const stab_opts *like, const std::string &name, int n,
                stab_path_choice *out) {
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess) e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return STAB_E_CUDA;
    }
    stab_path_choice c{};
    int rc = measure(device, like, n, &c);
    cudaSetDevice(prev);
    if (rc != STAB_OK) return rc;
    rc = stab_path_store(name.c_str(), n, &c);
    if (rc != STAB_OK) return rc;
    if (const char *p = cache_file()) {
        std::lock_guard<std::mutex> g(g_mu);
        write_file(p);
    }
    if (out) *out = c;
    return STAB_OK;
}

}  // namespace

int resolve_path_choice(int device, int n, const stab_opts *like, stab_path_choice *out) {
    std::string name;
    int rc = device_name(device, &name);
    if (rc != STAB_OK) return rc;
    if (stab_path_lookup(name.c_str(), n, out) == STAB_OK) return STAB_OK;
    if (!tuning_enabled()) return stab_path_defaults(n, out);
    // one tuning per (GPU, n) even when several threads create contexts at once
    std::lock_guard<std::mutex> g(g_tune_mu);
    if (stab_path_lookup(name.c_str(), n, out) == STAB_OK) return STAB_OK;
    return tune_locked(device, like, name, n, out);
}

}  // namespace stab

using namespace stab;

extern "C" {

int stab_path_defaults(int n, stab_path_choice *out) {
    if (!out) return STAB_E_INVAL;
    if (n < 1 || n > STAB_MAX_QUBITS) return STAB_E_RANGE;
    stab_path_choice c{};
    c.resident = 1;
    c.resident_adjoint = 1;
    c.gen_cut = n == 4 ? 0.56 : 0.5;
    c.tile_limit = (int64_t)1 << 17;
    c.tuned = 0;
    c.gen_parts = 2;
    *out = c;
    return STAB_OK;
}

int stab_path_lookup(const char *gpu_name, int n, stab_path_choice *out) {
    if (!gpu_name || !out) return STAB_E_INVAL;
    if (n < 1 || n > STAB_MAX_QUBITS) return STAB_E_RANGE;
    std::lock_guard<std::mutex> g(g_mu);
    read_env_file_locked();
    auto it = g_cache.find({std::string(gpu_name), n});
    if (it == g_cache.end()) return STAB_E_STATE;
    *out = it->second;
    return STAB_OK;
}

int stab_path_store(const char *gpu_name, int n, const stab_path_choice *choice) {
    if (!choice || !name_ok(gpu_name) || !choice_ok(*choice)) return STAB_E_INVAL;
    if (n < 1 || n > STAB_MAX_QUBITS) return STAB_E_RANGE;
    std::lock_guard<std::mutex> g(g_mu);
    read_env_file_locked();
    g_cache[{std::string(gpu_name), n}] = *choice;
    return STAB_OK;
}

int stab_path_clear(void) {
    std::lock_guard<std::mutex> g(g_mu);
    g_cache.clear();
    g_file_read = true;   // an explicit clear also forgets the environment's file
    return STAB_OK;
}

int stab_path_save(const char *path) {
    if (!path) return STAB_E_INVAL;
    std::lock_guard<std::mutex> g(g_mu);
    return write_file(path) ? STAB_OK : STAB_E_STATE;
}

int stab_path_load(const char *path) {
    if (!path) return STAB_E_INVAL;
    std::map<std::pair<std::string, int>, stab_path_choice> m;
    bool opened = false;
    if (!read_file(path, &m, &opened)) return STAB_E_INVAL;
    if (!opened) return STAB_E_STATE;
    std::lock_guard<std::mutex> g(g_mu);
    for (auto &kv : m) g_cache[kv.first] = kv.second;
    return STAB_OK;
}

int stab_path_tune(int device, int n, stab_path_choice *out) {
    if (n < 1 || n > STAB_MAX_QUBITS) return STAB_E_RANGE;
    std::string name;
    int rc = device_name(device, &name);
    if (rc != STAB_OK) return rc;
    std::lock_guard<std::mutex> g(g_tune_mu);
    return tune_locked(device, nullptr, name, n, out);
}

}  // extern "C"
