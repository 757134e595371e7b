// device_ops.cuh -- per-group and per-index gate actions used by every kernel.
//
// Layout: index(P) = z | (x << n); bit q is z_q, bit n+q is x_q.  The four
// strings that differ only on wire q form a group with slots
//   I = base, Z = base | 1<<q, X = base | 1<<(n+q), Y = X | Z,
// and a single-qubit gate on q maps each group to itself (Sec. II-A: only the
// j-th factor of each string changes).  In registers a group is held as
// (x, y, z) -- the I slot never changes.
#pragma once

#include <cstdint>

#include "stab_internal.h"

namespace stab {

// Sign flip by XOR of the sign bit: an integer operation, so signed
// permutations never touch the FP64 pipe and stay bit-exact.
__device__ __forceinline__ double flip(double v, uint32_t neg) {
    return __hiloint2double(__double2hiint(v) ^ (int)(neg << 31), __double2loint(v));
}

// Insert a zero bit at position p.
__device__ __forceinline__ uint64_t insert0(uint64_t v, int p) {
    uint64_t lo = v & ((1ull << p) - 1ull);
    return ((v >> p) << (p + 1)) | lo;
}

// Base index of group g on wire q: zeros at bits q (z_q) and n+q (x_q).
__device__ __forceinline__ uint64_t group_base(uint64_t g, int n, int q) {
    return insert0(insert0(g, q), n + q);
}

// Signed permutation code on the (X, Y, Z) slots: for output slot o = 0, 1, 2
// (X, Y, Z), bits [3o, 3o+1] hold the source slot (0, 1, 2) and bit 3o+2 the
// sign.
__device__ __forceinline__ void apply_perm(double &x, double &y, double &z, uint32_t code) {
    double in0 = x, in1 = y, in2 = z;
    uint32_t s0 = code & 3u, s1 = (code >> 3) & 3u, s2 = (code >> 6) & 3u;
    double o0 = s0 == 0 ? in0 : (s0 == 1 ? in1 : in2);
    double o1 = s1 == 0 ? in0 : (s1 == 1 ? in1 : in2);
    double o2 = s2 == 0 ? in0 : (s2 == 1 ? in1 : in2);
    x = flip(o0, (code >> 2) & 1u);
    y = flip(o1, (code >> 5) & 1u);
    z = flip(o2, (code >> 8) & 1u);
}

// Rotation of the pair (u, v) by the reduced angle phi (|phi| <= pi/2) with
// three shears (lifting): u += t v; v += s u; u += t v, t = -tan(phi/2),
// s = sin(phi).  Three FMAs per pair instead of the four products of the
// matrix form.  neg applies the factor R(pi) (u, v -> -u, -v) first.  The
// inverse rotation is the same with (t, s) -> (-t, -s).
__device__ __forceinline__ void lift(double &u, double &v, double t, double s, uint32_t neg) {
    u = flip(u, neg);
    v = flip(v, neg);
    u = fma(t, v, u);
    v = fma(s, u, v);
    u = fma(t, v, u);
}

__device__ __forceinline__ void apply_rot(double &x, double &y, double &z, int axis, double t,
                                          double s, uint32_t neg) {
    if (axis == AX_X) {
        lift(y, z, t, s, neg);
    } else if (axis == AX_Y) {
        lift(z, x, t, s, neg);
    } else {
        lift(x, y, t, s, neg);
    }
}

__device__ __forceinline__ void apply_map3(double &x, double &y, double &z, const double *m,
                                           bool transpose) {
    double a = x, b = y, c = z;
    if (!transpose) {
        x = fma(m[2], c, fma(m[1], b, m[0] * a));
        y = fma(m[5], c, fma(m[4], b, m[3] * a));
        z = fma(m[8], c, fma(m[7], b, m[6] * a));
    } else {
        x = fma(m[6], c, fma(m[3], b, m[0] * a));
        y = fma(m[7], c, fma(m[4], b, m[1] * a));
        z = fma(m[8], c, fma(m[5], b, m[2] * a));
    }
}

// One single-qubit op on a group held in registers; inverse = 1 applies its
// inverse (backward propagation).
__device__ __forceinline__ void apply_op1(double &x, double &y, double &z, const DevOp &op,
                                          const DevMap3 *maps, int inverse) {
    if (op.kind == K_ROT) {
        double t = inverse ? -op.t : op.t;
        double s = inverse ? -op.s : op.s;
        apply_rot(x, y, z, op.axis, t, s, op.perm);
    } else if (op.kind == K_PERM) {
        apply_perm(x, y, z, inverse ? op.perm_inv : op.perm);
    } else {  // K_MAP3
        apply_map3(x, y, z, maps[op.param].m, inverse != 0);
    }
}

// Source index and sign of output index i under one two-qubit Clifford (pull
// form).  Both index maps are involutions and both sign rules are invariant
// under them, so forward and inverse differ only in the order of traversal.
//   CX(c -> t): x_t ^= x_c, z_c ^= z_t; minus iff x_c & z_t & !(x_t ^ z_c)
//     (the map_CX list of Sec. III-C, XZ <-> -YY);
//   CZ(a, b):   z_a ^= x_b, z_b ^= x_a; minus iff x_a & x_b & (z_a ^ z_b).
__device__ __forceinline__ uint64_t pull_2q_ab(uint64_t i, int n, bool is_cx, int a, int b,
                                               uint32_t &neg) {
    if (is_cx) {
        uint64_t xc = (i >> (n + a)) & 1ull, zt = (i >> b) & 1ull;
        uint64_t j = i ^ (xc << (n + b)) ^ (zt << a);
        uint32_t xt = (uint32_t)((j >> (n + b)) & 1ull), zc = (uint32_t)((j >> a) & 1ull);
        neg ^= (uint32_t)(xc & zt) & (1u ^ (xt ^ zc));
        return j;
    } else {
        uint64_t xa = (i >> (n + a)) & 1ull, xb = (i >> (n + b)) & 1ull;
        uint64_t j = i ^ (xb << a) ^ (xa << b);
        uint32_t za = (uint32_t)((j >> a) & 1ull), zb = (uint32_t)((j >> b) & 1ull);
        neg ^= (uint32_t)(xa & xb) & (za ^ zb);
        return j;
    }
}

__device__ __forceinline__ uint64_t pull_2q(uint64_t i, int n, const DevOp &op, uint32_t &neg) {
    return pull_2q_ab(i, n, op.kind == K_CX, op.q, op.q1, neg);
}

// 32-bit forms for the resident kernels (an index has at most 2n <= 24 bits).
__device__ __forceinline__ uint32_t insert0_32(uint32_t v, int p) {
    return ((v >> p) << (p + 1)) | (v & ((1u << p) - 1u));
}

__device__ __forceinline__ uint32_t group_base32(uint32_t g, int n, int q) {
    return insert0_32(insert0_32(g, q), n + q);
}

__device__ __forceinline__ uint32_t pull_2q_32(uint32_t i, int n, bool is_cx, int a, int b,
                                               uint32_t &neg) {
    if (is_cx) {
        const uint32_t xc = (i >> (n + a)) & 1u, zt = (i >> b) & 1u;
        const uint32_t j = i ^ (xc << (n + b)) ^ (zt << a);
        neg ^= xc & zt & (1u ^ (((j >> (n + b)) ^ (j >> a)) & 1u));
        return j;
    } else {
        const uint32_t xa = (i >> (n + a)) & 1u, xb = (i >> (n + b)) & 1u;
        const uint32_t j = i ^ (xb << a) ^ (xa << b);
        neg ^= xa & xb & (((j >> a) ^ (j >> b)) & 1u);
        return j;
    }
}

// Source of output index i through the pull records of a stream pass (stored
// in pull order).
__device__ __forceinline__ uint32_t pull_recs(uint32_t i, int n, const Rec *pulls, int n_pull,
                                              uint32_t &neg) {
    for (int k = 0; k < n_pull; ++k) {
        const Rec &p = pulls[k];
        i = pull_2q_32(i, n, p.kind == R_CX, p.q, p.q1, neg);
    }
    return i;
}

// Applies the op records of a stream pass to a group held in registers.
__device__ __forceinline__ void apply_recs(double &x, double &y, double &z, const Rec *ops,
                                           int n_recs) {
    for (int k = 0; k < n_recs; ++k) {
        const Rec &op = ops[k];
        if (op.kind == R_ROT) {
            apply_rot(x, y, z, op.axis, op.t, op.s, op.code);
        } else if (op.kind == R_PERM) {
            apply_perm(x, y, z, op.code);
        } else if (op.kind == R_MAP3) {
            apply_map3(x, y, z, reinterpret_cast<const double *>(&ops[k + 1]), false);
            k += 3;
        }
    }
}

// Source of output index i through a whole P_CLIFF pass.  Forward: the ops
// were applied first to last, so the pull walks them last to first; the
// inverse pass applies the inverses last to first, so its pull walks first to
// last.
__device__ __forceinline__ uint64_t pull_pass(uint64_t i, int n, const DevOp *ops, int n_ops,
                                              int inverse, uint32_t &neg) {
    if (!inverse) {
        for (int k = n_ops - 1; k >= 0; --k) i = pull_2q(i, n, ops[k], neg);
    } else {
        for (int k = 0; k < n_ops; ++k) i = pull_2q(i, n, ops[k], neg);
    }
    return i;
}

}  // namespace stab
