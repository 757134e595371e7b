// noalloc.cu -- expectation values without any device allocation.
//
// Some callers cannot allocate device memory at all: a host program that
// reserves its whole device budget at start-up and forbids growth afterwards,
// code that runs inside another framework whose allocator owns every byte of
// the device, or a path that must not risk an out-of-memory failure halfway.
// stab_expect_static serves them: it runs the streamed expectation path
// (the same kernels as stab_expect with STAB_KERNEL_STREAMED) on a fixed
// workspace that the library declares as a file-scope __device__ array, so it
// calls no cudaMalloc, cudaFree or other allocating routine.
//
// The workspace (kStaticBytes) is reserved on every GPU that loads the
// library, for as long as the library stays loaded.  All calls share it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/stab.h"
#include "launch.h"
#include "planner.h"

namespace stab {

namespace {

constexpr size_t kStaticBytes = 16ull << 20;   // 16 MiB

// The workspace.  Host code must not pass this name to a kernel: on the host
// it is only a stand-in symbol, not the device address.
static __device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

std::mutex g_ws_mu;
void *g_ws_addr[64] = {};

// Device address of the workspace on the current device, looked up once per
// device (with that device current) by the first call on it.  The address
// is cached for the life of the process: a cudaDeviceReset() recreates the
// device's context and leaves the cached address stale, so this entry point
// is not supported after a reset of a device it has already run on.
int workspace_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return STAB_E_CUDA;
    }
    if (dev < 0 || dev >= 64) return STAB_E_RANGE;
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if (!g_ws_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess || p == nullptr) {
            record_cuda_error(e);
            return STAB_E_CUDA;
        }
        g_ws_addr[dev] = p;
    }
    *out = g_ws_addr[dev];
    return STAB_OK;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

}  // namespace stab

using namespace stab;

extern "C" int stab_expect_static(int n, const stab_gate *gates, int64_t m, const double *thetas,
                                  int64_t n_params, const stab_term *O, int64_t n_terms,
                                  double *out, void *stream) {
    if (!out) return STAB_E_INVAL;
    if (n < 1 || n > STAB_MAX_QUBITS) return STAB_E_RANGE;
    int rc = validate_gates(n, gates, m, n_params, nullptr);
    if (rc != STAB_OK) return rc;
    rc = validate_thetas(thetas, n_params);
    if (rc != STAB_OK) return rc;
    std::vector<DevTerm> terms;
    rc = encode_terms(n, O, n_terms, &terms);
    if (rc != STAB_OK) return rc;

    HostPlan P;
    build_plan(n, gates, m, n_params, PLAN_FUSED, &P);

    // workspace layout: ops | maps | map gate indices | raw gates | angles |
    // terms | result | vector A | vector B
    const size_t vec = sizeof(double) << (2 * n);
    const size_t b_ops = up256(P.ops.size() * sizeof(DevOp));
    const size_t b_maps = up256(P.maps.size() * sizeof(DevMap3));
    const size_t b_midx = up256(P.map_gate_idx.size() * sizeof(int32_t));
    const size_t b_raw = up256(P.raw.size() * sizeof(RawGate));
    const size_t b_th = up256((size_t)(n_params > 0 ? n_params : 1) * sizeof(double));
    const size_t b_terms = up256((terms.size() ? terms.size() : 1) * sizeof(DevTerm));
    const size_t b_res = 256;
    const size_t total = b_ops + b_maps + b_midx + b_raw + b_th + b_terms + b_res + 2 * vec;
    if (total > kStaticBytes) return STAB_E_RANGE;   // does not fit the 16 MiB workspace

    cudaStream_t s = (cudaStream_t)stream;
    // the workspace is the current device's; a stream of another device
    // would run these kernels against a pointer it cannot use
    if (s != nullptr) {
        int cur_dev = 0, st_dev = 0;
        cudaError_t de = cudaGetDevice(&cur_dev);
        if (de == cudaSuccess) de = cudaStreamGetDevice(s, &st_dev);
        if (de != cudaSuccess) {
            record_cuda_error(de);
            return STAB_E_CUDA;
        }
        if (st_dev != cur_dev) return STAB_E_INVAL;
    }
    void *ws = nullptr;
    rc = workspace_address(&ws);
    if (rc != STAB_OK) return rc;
    char *base = (char *)ws;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        char *p = base + off;
        off += bytes;
        return p;
    };
    DevOp *d_ops = (DevOp *)carve(b_ops);
    DevMap3 *d_maps = (DevMap3 *)carve(b_maps);
    int32_t *d_midx = (int32_t *)carve(b_midx);
    RawGate *d_raw = (RawGate *)carve(b_raw);
    double *d_th = (double *)carve(b_th);
    DevTerm *d_terms = (DevTerm *)carve(b_terms);
    double *d_res = (double *)carve(b_res);
    double *vA = (double *)carve(vec);
    double *vB = (double *)carve(vec);

    auto h2d = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        if (!bytes) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    cudaError_t e = h2d(d_ops, P.ops.data(), P.ops.size() * sizeof(DevOp));
    if (e == cudaSuccess) e = h2d(d_maps, P.maps.data(), P.maps.size() * sizeof(DevMap3));
    if (e == cudaSuccess) e = h2d(d_midx, P.map_gate_idx.data(), P.map_gate_idx.size() * 4);
    if (e == cudaSuccess) e = h2d(d_raw, P.raw.data(), P.raw.size() * sizeof(RawGate));
    if (e == cudaSuccess) e = h2d(d_th, thetas, (size_t)n_params * sizeof(double));
    if (e == cudaSuccess) e = h2d(d_terms, terms.data(), terms.size() * sizeof(DevTerm));
    if (e == cudaSuccess && (!P.ops.empty() || !P.maps.empty()))
        e = launch_encode(d_ops, (int)P.ops.size(), d_maps, (int)P.maps.size(),
                          max_map_count(P.maps.data(), P.maps.size()), d_midx, d_raw, d_th, s);
    // every entry of the working vector is written here, so nothing left by
    // an earlier call survives
    if (e == cudaSuccess)
        e = launch_fill(vA, n, 1, INIT_TERMS, d_terms, (int)terms.size(), s);
    double *cur = vA, *alt = vB;
    const int np = (int)P.passes.size();
    for (int k = np - 1; k >= 0 && e == cudaSuccess; --k) {
        const DevPass &p = P.passes[k];
        if (p.type == P_WIRE) {
            e = launch_stream_wire(cur, n, 1, p, d_ops, d_maps, 1, s);
        } else {
            e = launch_stream_cliff(cur, alt, n, 1, p, d_ops, 1, s);
            double *t = cur;
            cur = alt;
            alt = t;
        }
    }
    if (e == cudaSuccess) e = launch_xfree_sum(cur, n, 1, d_res, s);
    double h = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_res, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return STAB_E_CUDA;
    }
    *out = h;
    return STAB_OK;
}
