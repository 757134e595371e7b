// k_sparse.cu -- propagation of a Pauli-term list: the sparse (lambda, I)
// representation of a stabilizer (Sec. II-B), kept while its stabilizer
// order n' (the number of strings, Fig. 1) is small, so that n is limited by
// the list, not by a 4^n vector (keys z | x << n in 64 bits, n <= 32).
//
// A run of Clifford gates maps every term in place: one signed string each
// (Table I rows H and S, the map_CX list, and their compositions).  A rotation
// R_sigma on wire q mixes the two strings of each anticommuting pair (u, v)
// -- R_x: (Y, Z), R_y: (Z, X), R_z: (X, Y) -- as u' = c u - s v,
// v' = s u + c v (Table I); a term whose partner is absent spawns it.  One
// rotation is four launches:
//   insert -- every anticommuting term claims a slot of an open-addressing
//             table (keys are unique, so a claim never meets its own key);
//   count  -- per term: the partner's position (or -1) and how many nonzero
//             terms it emits; per block: the total;
//   scan   -- one CTA: exclusive scan of the block totals, the new order,
//             capacity and threshold checks;
//   write  -- every term writes its images at their scanned positions (in
//             input order, so the list order is deterministic and independent
//             of the grid) and frees its table slot.
// Exact zeros are never stored.  A step that finds the stop flag set by an
// earlier step returns at once, so the host can launch several steps ahead.
#include <cuda_runtime.h>

#include "../../include/stab.h"
#include "launch.h"

namespace stab {

namespace {

constexpr int kSpThreads = 256;

// letter code 2x + z: I = 0, Z = 1, X = 2, Y = 3
__device__ __forceinline__ uint32_t sp_letter(uint64_t key, int n, int q) {
    return (uint32_t)(((key >> (n + q)) & 1u) << 1) | (uint32_t)((key >> q) & 1u);
}

__device__ __forceinline__ uint64_t sp_with_letter(uint64_t key, int n, int q, uint32_t lc) {
    key &= ~((1ull << q) | (1ull << (n + q)));
    return key | ((uint64_t)(lc & 1u) << q) | ((uint64_t)(lc >> 1) << (n + q));
}

// the anticommuting pair (u, v) of each rotation axis
__device__ __forceinline__ void sp_pair(int axis, uint32_t &u, uint32_t &v) {
    if (axis == 0) { u = 3u; v = 1u; }        // R_x: (Y, Z)
    else if (axis == 1) { u = 1u; v = 2u; }   // R_y: (Z, X)
    else { u = 2u; v = 3u; }                  // R_z: (X, Y)
}

__device__ __forceinline__ uint32_t sp_hash(uint64_t key, int log_h) {
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - log_h));
}

// Steps run until a stop: flags[0] != 0 at step flags[1].
__device__ __forceinline__ bool sp_stopped_before(const int32_t *flags, int step) {
    return flags[0] != 0 && flags[1] < step;
}

// Forward conjugation g P g^dagger of one Clifford gate on a key; sets the
// sign bit in neg.  1q rules on (x, z) of the wire: H swaps x and z (Y -> -Y),
// S: z ^= x (Y -> -X), S^dagger: z ^= x (X -> -Y), X: sign z, Y: sign x ^ z,
// Z: sign x.  CX(c, t): x_t ^= x_c, z_c ^= z_t, minus iff x_c z_t (x_t == z_c);
// CZ(a, b): z_a ^= x_b, z_b ^= x_a, minus iff x_a x_b (z_a != z_b).
__device__ __forceinline__ uint64_t sp_clifford(uint64_t key, int n, const SpGate g,
                                                uint32_t &neg) {
    const int a = g.q0;
    const uint32_t xa = (uint32_t)(key >> (n + a)) & 1u, za = (uint32_t)(key >> a) & 1u;
    switch (g.op) {
    case STAB_H:
        neg ^= xa & za;
        return sp_with_letter(key, n, a, (za << 1) | xa);
    case STAB_S:
        neg ^= xa & za;
        return sp_with_letter(key, n, a, (xa << 1) | (za ^ xa));
    case STAB_SDG:
        neg ^= xa & (za ^ 1u);
        return sp_with_letter(key, n, a, (xa << 1) | (za ^ xa));
    case STAB_X: neg ^= za; return key;
    case STAB_Y: neg ^= xa ^ za; return key;
    case STAB_Z: neg ^= xa; return key;
    case STAB_CX: {
        const int t = g.q1;
        const uint32_t xt = (uint32_t)(key >> (n + t)) & 1u, zt = (uint32_t)(key >> t) & 1u;
        neg ^= xa & zt & ((xt ^ za) ^ 1u);
        key = sp_with_letter(key, n, t, ((xt ^ xa) << 1) | zt);
        return sp_with_letter(key, n, a, (xa << 1) | (za ^ zt));
    }
    case STAB_CZ: {
        const int b = g.q1;
        const uint32_t xb = (uint32_t)(key >> (n + b)) & 1u, zb = (uint32_t)(key >> b) & 1u;
        neg ^= xa & xb & (za ^ zb);
        key = sp_with_letter(key, n, a, (xa << 1) | (za ^ xb));
        return sp_with_letter(key, n, b, (xb << 1) | (zb ^ xa));
    }
    default: return key;
    }
}

__device__ __forceinline__ void sp_block_range(int64_t count, int64_t &lo, int64_t &hi) {
    const int64_t per = (count + gridDim.x - 1) / gridDim.x;
    lo = (int64_t)blockIdx.x * per;
    if (lo > count) lo = count;
    hi = lo + per;
    if (hi > count) hi = count;
}

// The images of term i under the rotation: up to two (key, value) pairs in the
// order u, v.  partner = position of the other string of the pair, or -1.
__device__ __forceinline__ int sp_images(uint64_t key, double val, int32_t partner,
                                         const double *vals, int n, int q, int axis, double c,
                                         double s, uint64_t &k0, double &v0, uint64_t &k1,
                                         double &v1) {
    uint32_t u, v;
    sp_pair(axis, u, v);
    const uint32_t L = sp_letter(key, n, q);
    if (L != u && L != v) {
        k0 = key;
        v0 = val;
        return 1;
    }
    double uu, vv;
    if (L == u) {
        uu = val;
        vv = partner >= 0 ? vals[partner] : 0.0;
    } else {
        if (partner >= 0) return 0;   // the u term of the pair writes both
        uu = 0.0;
        vv = val;
    }
    const double ou = fma(c, uu, -(s * vv));
    const double ov = fma(s, uu, c * vv);
    const uint64_t ku = sp_with_letter(key, n, q, u), kv = sp_with_letter(key, n, q, v);
    int e = 0;
    if (ou != 0.0) { k0 = ku; v0 = ou; e = 1; }
    if (ov != 0.0) {
        if (e == 0) { k0 = kv; v0 = ov; }
        else { k1 = kv; v1 = ov; }
        ++e;
    }
    return e;
}

template <typename T>
__device__ T block_exclusive_scan(T x, T &total, T *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (int)(blockDim.x >> 5) ? sh[lane] : (T)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;   // inclusive prefix over warps
    }
    __syncthreads();
    const T warp_before = warp > 0 ? sh[warp - 1] : (T)0;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_before + incl - x;
}

// cos and sin of a slot's angle, from the table k_sp_cos_sin fills once per
// circuit load (cs[2 p] = cos, cs[2 p + 1] = sin): every thread of every block
// needs them, and evaluating sincos there cost the FP64 pipe more than the
// rotation itself on short lists.
__device__ __forceinline__ void sp_rot_cs(const double *cs, int param, int inverse, double &c,
                                          double &s) {
    c = cs[2 * param];
    s = cs[2 * param + 1];
    if (inverse) s = -s;
}

__global__ void k_sp_cos_sin(const double *thetas, int64_t n_params, double *cs) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_params) sincos(thetas[p], &cs[2 * p + 1], &cs[2 * p]);
}

__global__ void __launch_bounds__(kSpThreads) k_sp_cliff(uint64_t *keys, double *vals,
                                                          int64_t *counts, const int32_t *flags,
                                                          int step, int n, const SpGate *gates,
                                                          int n_gates) {
    if (sp_stopped_before(flags, step)) return;
    const int64_t count = counts[step];
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[step + 1] = count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        uint32_t neg = 0;
        for (int g = 0; g < n_gates; ++g) k = sp_clifford(k, n, gates[g], neg);
        keys[i] = k;
        if (neg) vals[i] = -vals[i];
    }
}

// A long Clifford run as its tableau: the images U X_q U^dagger and
// U Z_q U^dagger of the 2n single-qubit generators (entry q: X_q, entry n + q:
// Z_q), each a signed string.  One thread per generator, gate by gate.
__global__ void k_sp_tableau(const SpGate *gates, const int32_t *run_first,
                             const int32_t *run_count, int n, SpTab *tabs) {
    const int r = blockIdx.x, j = threadIdx.x;
    if (j >= 2 * n) return;
    uint64_t k = j < n ? (1ull << (n + j)) : (1ull << (j - n));
    uint32_t neg = 0;
    const SpGate *g = gates + run_first[r];
    for (int i = 0; i < run_count[r]; ++i) k = sp_clifford(k, n, g[i], neg);
    tabs[(size_t)r * 64 + j] = SpTab{k, neg};
}

// Exponent c (mod 4) of P(a) P(b) = i^c P(a xor b) for Hermitian Pauli strings
// given by x / z masks: per qubit, with a = Y: z_b - x_b; a = X: z_b (2 x_b - 1);
// a = Z: x_b (1 - 2 z_b) (the phase function of the stabilizer tableau
// algorithm of Aaronson and Gottesman), summed with population counts.
__device__ __forceinline__ uint32_t sp_mul_phase(uint32_t ax, uint32_t az, uint32_t bx,
                                                 uint32_t bz) {
    const uint32_t A = ax & az, B = ax & ~az, C = ~ax & az;
    const uint32_t plus = (A & bz & ~bx) | (B & bz & bx) | (C & bx & ~bz);
    const uint32_t minus = (A & bx & ~bz) | (B & bz & ~bx) | (C & bx & bz);
    return (uint32_t)(__popc(plus) - __popc(minus)) & 3u;
}

// The tableau regrouped by chunks of kSpChunkQubits qubits: entry
// (chunk c, subset t) is the ordered product prod_{q in c} (U X_q U^dagger)^{x_q}
// (U Z_q U^dagger)^{z_q} of the generator images the subset selects (bit j of
// t: x of qubit 4c + j, bit 4 + j: its z), as a Hermitian string and a phase
// i^e.  One block per (run, chunk), one thread per subset.
__global__ void k_sp_tab_chunks(const SpTab *tabs, int n, SpChunk *chunks) {
    const int r = blockIdx.x / kSpChunks, c = blockIdx.x % kSpChunks, t = threadIdx.x;
    const uint64_t zmask = (1ull << n) - 1;
    uint32_t rx = 0, rz = 0, e = 0;
    for (int j = 0; j < kSpChunkQubits; ++j) {
        const int q = kSpChunkQubits * c + j;
        if (q >= n) break;
        for (int part = 0; part < 2; ++part) {   // X_q, then Z_q
            if (!((t >> (part * kSpChunkQubits + j)) & 1)) continue;
            const SpTab g = tabs[(size_t)r * 64 + (part ? n + q : q)];
            const uint32_t gx = (uint32_t)(g.key >> n), gz = (uint32_t)(g.key & zmask);
            e += sp_mul_phase(rx, rz, gx, gz) + (g.neg ? 2u : 0u);
            rx ^= gx;
            rz ^= gz;
        }
    }
    chunks[(size_t)blockIdx.x * 256 + t] = SpChunk{rx, rz, e & 3u, 0u};
}

// U P U^dagger from the tableau: P(x, z) = i^{|x & z|} prod_q X_q^{x_q} Z_q^{z_q}
// (Y = i X Z), so its image is i^{|x & z|} times the product of the generator
// images in that order, each factor adding its phase and sign.  The product
// is taken chunk by chunk from the run's chunk table (staged in shared
// memory): ceil(n / 4) lookups and string products per term instead of one
// product per set bit.
__global__ void __launch_bounds__(kSpThreads) k_sp_cliff_tab(uint64_t *keys, double *vals,
                                                              int64_t *counts,
                                                              const int32_t *flags, int step,
                                                              int n, const SpChunk *chunks) {
    __shared__ SpChunk sc[kSpChunks * 256];
    if (sp_stopped_before(flags, step)) return;
    const int n_ch = (n + kSpChunkQubits - 1) / kSpChunkQubits;
    for (int k = threadIdx.x; k < n_ch * 256; k += blockDim.x) sc[k] = chunks[k];
    __syncthreads();
    const int64_t count = counts[step];
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[step + 1] = count;
    const uint64_t zmask = (1ull << n) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        const uint32_t x = (uint32_t)(k >> n), z = (uint32_t)(k & zmask);
        uint32_t rx = 0, rz = 0, e = (uint32_t)__popc(x & z);
        for (int c = 0; c < n_ch; ++c) {
            const uint32_t sh = (uint32_t)(kSpChunkQubits * c);
            const SpChunk g = sc[c * 256 + (((x >> sh) & 15u) | (((z >> sh) & 15u) << 4))];
            e += g.e + sp_mul_phase(rx, rz, g.x, g.z);
            rx ^= g.x;
            rz ^= g.z;
        }
        // a Hermitian image: e is 0 or 2 (mod 4)
        keys[i] = ((uint64_t)rx << n) | rz;
        if (e & 2u) vals[i] = -vals[i];
    }
}

__global__ void __launch_bounds__(kSpThreads) k_sp_insert(const uint64_t *keys,
                                                           const int64_t *counts,
                                                           const int32_t *flags, int step, int n,
                                                           int q, int axis, SpSlot *table,
                                                           int log_h,
                                                           int32_t *slot_of, int32_t *err) {
    if (sp_stopped_before(flags, step)) return;
    const int64_t count = counts[step];
    uint32_t u, v;
    sp_pair(axis, u, v);
    const uint32_t mask = (1u << log_h) - 1u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        const uint32_t L = sp_letter(k, n, q);
        if (L != u && L != v) continue;
        uint32_t s = sp_hash(k, log_h);
        // the table is at least twice the list, so a free slot is near; the
        // bound only guards against a corrupted table
        bool ok = false;
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            if (atomicCAS(&table[s].pos, -1, (int32_t)i) == -1) {
                table[s].key = k;
                slot_of[i] = (int32_t)s;
                ok = true;
                break;
            }
            s = (s + 1u) & mask;
        }
        if (!ok) {
            slot_of[i] = -1;
            atomicExch(err, 1);
        }
    }
}

__device__ __forceinline__ int32_t sp_lookup(uint64_t k, const SpSlot *table, int log_h) {
    const uint32_t mask = (1u << log_h) - 1u;
    uint32_t s = sp_hash(k, log_h);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        // one 16-byte load: key and position of the slot
        const ulonglong2 e = *reinterpret_cast<const ulonglong2 *>(table + s);
        const int32_t p = (int32_t)(uint32_t)e.y;
        if (p < 0) return -1;
        if (e.x == k) return p;
        s = (s + 1u) & mask;
    }
    return -1;
}

__global__ void __launch_bounds__(kSpThreads) k_sp_count(const uint64_t *keys,
                                                          const double *vals,
                                                          const int64_t *counts,
                                                          const int32_t *flags, int step, int n,
                                                          int q, int axis, const double *cs,
                                                          int param, int inverse,
                                                          const SpSlot *table, int log_h,
                                                          int32_t *partner, int64_t *blk) {
    __shared__ int64_t sh[32];
    if (sp_stopped_before(flags, step)) return;
    const int64_t count = counts[step];
    int64_t lo, hi;
    sp_block_range(count, lo, hi);
    double c, s;
    sp_rot_cs(cs, param, inverse, c, s);
    uint32_t u, v;
    sp_pair(axis, u, v);
    int64_t mine = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint64_t k = keys[i];
        const uint32_t L = sp_letter(k, n, q);
        int32_t p = -1;
        if (L == u || L == v) {
            p = sp_lookup(sp_with_letter(k, n, q, L == u ? v : u), table, log_h);
            partner[i] = p;
        }
        uint64_t k0, k1;
        double v0, v1;
        mine += sp_images(k, vals[i], p, vals, n, q, axis, c, s, k0, v0, k1, v1);
    }
    int64_t total;
    (void)block_exclusive_scan<int64_t>(mine, total, sh);
    if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

// One CTA of 1024 threads: exclusive scan of nblk <= 1024 block totals.
__global__ void __launch_bounds__(1024) k_sp_scan(int64_t *blk, int nblk, int64_t *counts,
                                                  int32_t *flags, int step, int64_t cap,
                                                  int64_t threshold) {
    __shared__ int64_t sh[32];
    if (sp_stopped_before(flags, step)) return;
    const int64_t x = (int)threadIdx.x < nblk ? blk[threadIdx.x] : 0;
    int64_t total;
    const int64_t ex = block_exclusive_scan<int64_t>(x, total, sh);
    if ((int)threadIdx.x < nblk) blk[threadIdx.x] = ex;
    if (threadIdx.x == 0) {
        if (total > cap) {
            flags[0] = 1;          // overflow: the step is not applied
            flags[1] = step;
        } else {
            counts[step + 1] = total;
            if (threshold > 0 && total > threshold) {
                flags[0] = 2;      // order above the threshold after this step
                flags[1] = step;
            }
        }
    }
}

__global__ void __launch_bounds__(kSpThreads) k_sp_write(
    const uint64_t *keys, const double *vals, const int64_t *counts, const int32_t *flags,
    int step, int n, int q, int axis, const double *cs, int param, int inverse,
    SpSlot *table, const int32_t *slot_of, const int32_t *partner, const int64_t *blk,
    uint64_t *keys_out, double *vals_out) {
    __shared__ int64_t sh[32];
    if (sp_stopped_before(flags, step)) return;
    if (flags[0] == 1 && flags[1] == step) return;
    const int64_t count = counts[step];
    int64_t lo, hi;
    sp_block_range(count, lo, hi);
    double c, s;
    sp_rot_cs(cs, param, inverse, c, s);
    uint32_t u, v;
    sp_pair(axis, u, v);
    int64_t base = blk[blockIdx.x];
    for (int64_t t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int64_t i = t0 + threadIdx.x;
        uint64_t k0 = 0, k1 = 0;
        double v0 = 0.0, v1 = 0.0;
        int e = 0;
        if (i < hi) {
            const uint64_t k = keys[i];
            const uint32_t L = sp_letter(k, n, q);
            int32_t p = -1;
            if (L == u || L == v) {
                p = partner[i];
                const int32_t slot = slot_of[i];
                if (slot >= 0) table[slot].pos = -1;
            }
            e = sp_images(k, vals[i], p, vals, n, q, axis, c, s, k0, v0, k1, v1);
        }
        int64_t tile_total;
        const int64_t at = base + block_exclusive_scan<int64_t>(e, tile_total, sh);
        if (e > 0) {
            keys_out[at] = k0;
            vals_out[at] = v0;
        }
        if (e > 1) {
            keys_out[at + 1] = k1;
            vals_out[at + 1] = v1;
        }
        base += tile_total;
    }
}

// Fixed-order sum of the coefficients of the x-free strings (x = key >> n == 0).
__global__ void __launch_bounds__(kSpThreads) k_sp_xfree(const uint64_t *keys,
                                                          const double *vals,
                                                          const int64_t *counts, int step,
                                                          int n, double *partial) {
    __shared__ double red[kSpThreads / 32];
    const int64_t count = counts[step];
    int64_t lo, hi;
    sp_block_range(count, lo, hi);
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
        if ((keys[i] >> n) == 0) acc += vals[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kSpThreads / 32; ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// One warp: lane l sums a contiguous slice of the partials, then a fixed
// shuffle tree; the order depends only on nblk.
__global__ void k_sp_sum_partials(const double *partial, int nblk, double *out) {
    const int lane = threadIdx.x;
    const int per = (nblk + 31) / 32;
    double t = 0.0;
    for (int b = lane * per; b < nblk && b < (lane + 1) * per; ++b) t += partial[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) *out = t;
}

__global__ void k_sp_to_terms(const uint64_t *keys, const double *vals, const int64_t *counts,
                              int step, DevTerm *out) {
    const int64_t count = counts[step];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = DevTerm{vals[i], keys[i]};
}

int sp_grid(int64_t bound) {
    int64_t b = (bound + 2047) / 2048;
    if (b < 1) b = 1;
    if (b > kSpMaxBlocks) b = kSpMaxBlocks;
    return (int)b;
}

}  // namespace

cudaError_t launch_sp_cos_sin(const double *thetas, int64_t n_params, double *cs,
                              cudaStream_t st) {
    if (n_params <= 0) return cudaSuccess;
    k_sp_cos_sin<<<(unsigned)((n_params + 255) / 256), 256, 0, st>>>(thetas, n_params, cs);
    return cudaGetLastError();
}

cudaError_t launch_sp_cliff(uint64_t *keys, double *vals, int64_t *counts, const int32_t *flags,
                            int step, int n, const SpGate *gates, int n_gates, int64_t bound,
                            cudaStream_t st) {
    k_sp_cliff<<<sp_grid(bound), kSpThreads, 0, st>>>(keys, vals, counts, flags, step, n, gates,
                                                        n_gates);
    return cudaGetLastError();
}

cudaError_t launch_sp_tableau(const SpGate *gates, const int32_t *run_first,
                              const int32_t *run_count, int n_runs, int n, SpTab *tabs,
                              SpChunk *chunks, cudaStream_t st) {
    if (n_runs == 0) return cudaSuccess;
    k_sp_tableau<<<n_runs, 64, 0, st>>>(gates, run_first, run_count, n, tabs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sp_tab_chunks<<<n_runs * kSpChunks, 256, 0, st>>>(tabs, n, chunks);
    return cudaGetLastError();
}

cudaError_t launch_sp_cliff_tab(uint64_t *keys, double *vals, int64_t *counts,
                                const int32_t *flags, int step, int n, const SpChunk *chunks,
                                int64_t bound, cudaStream_t st) {
    k_sp_cliff_tab<<<sp_grid(bound), kSpThreads, 0, st>>>(keys, vals, counts, flags, step, n,
                                                           chunks);
    return cudaGetLastError();
}

cudaError_t launch_sp_rotation(const SpRotArgs &a, cudaStream_t st) {
    const int grid = sp_grid(a.bound);
    k_sp_insert<<<grid, kSpThreads, 0, st>>>(a.keys, a.counts, a.flags, a.step, a.n, a.q,
                                              a.axis, a.table, a.log_h, a.slot_of,
                                              a.err);
    k_sp_count<<<grid, kSpThreads, 0, st>>>(a.keys, a.vals, a.counts, a.flags, a.step, a.n, a.q,
                                             a.axis, a.cs, a.param, a.inverse, a.table,
                                             a.log_h, a.partner, a.blk);
    k_sp_scan<<<1, 1024, 0, st>>>(a.blk, grid, a.counts, a.flags, a.step, a.cap, a.threshold);
    k_sp_write<<<grid, kSpThreads, 0, st>>>(a.keys, a.vals, a.counts, a.flags, a.step, a.n, a.q,
                                             a.axis, a.cs, a.param, a.inverse, a.table,
                                             a.slot_of, a.partner, a.blk, a.keys_out,
                                             a.vals_out);
    return cudaGetLastError();
}

cudaError_t launch_sp_xfree(const uint64_t *keys, const double *vals, const int64_t *counts,
                            int step, int n, double *partial, double *out, cudaStream_t st) {
    k_sp_xfree<<<kSpMaxBlocks, kSpThreads, 0, st>>>(keys, vals, counts, step, n, partial);
    k_sp_sum_partials<<<1, 32, 0, st>>>(partial, kSpMaxBlocks, out);
    return cudaGetLastError();
}

cudaError_t launch_sp_to_terms(const uint64_t *keys, const double *vals, const int64_t *counts,
                               int step, DevTerm *out, int64_t bound, cudaStream_t st) {
    k_sp_to_terms<<<sp_grid(bound), kSpThreads, 0, st>>>(keys, vals, counts, step, out);
    return cudaGetLastError();
}

}  // namespace stab
