// planner.cpp -- host-side validation, gate encoding and pass planning (see planner.h).
#include "planner.h"

#include "host_pool.h"
#include "launch.h"

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <cmath>
#include <map>

namespace stab {

// Gate lists of at least this many gates are planned in kPlanChunks chunks at
// once (see build_plan).
constexpr int64_t kParallelPlanGates = 16384;
constexpr int kPlanChunks = 8;

namespace {

bool is_two_qubit(int op) { return op == STAB_CX || op == STAB_CZ; }
bool is_rotation(int op) { return op == STAB_RX || op == STAB_RY || op == STAB_RZ; }

uint32_t make_perm(int s0, int n0, int s1, int n1, int s2, int n2) {
    return (uint32_t)(s0 | (n0 << 2) | (s1 << 3) | (n1 << 5) | (s2 << 6) | (n2 << 8));
}

}  // namespace

// Slots 0, 1, 2 = X, Y, Z; new[o] = (-1)^neg old[src] (Table I rows H and S;
// S^dagger, X, Y, Z are the standard conjugations).
uint32_t clifford_perm_code(int op) {
    switch (op) {
    case STAB_H: return make_perm(2, 0, 1, 1, 0, 0);    // X <- Z, Y <- -Y, Z <- X
    case STAB_S: return make_perm(1, 1, 0, 0, 2, 0);    // X <- -Y, Y <- X
    case STAB_SDG: return make_perm(1, 0, 0, 1, 2, 0);  // X <- Y, Y <- -X
    case STAB_X: return make_perm(0, 0, 1, 1, 2, 1);    // Y, Z negated
    case STAB_Y: return make_perm(0, 1, 1, 0, 2, 1);    // X, Z negated
    case STAB_Z: return make_perm(0, 1, 1, 1, 2, 0);    // X, Y negated
    default: return kPermIdentity;
    }
}

uint32_t perm_compose(uint32_t first, uint32_t then) {
    uint32_t out = 0;
    for (int o = 0; o < 3; ++o) {
        uint32_t s2 = (then >> (3 * o)) & 3u, n2 = (then >> (3 * o + 2)) & 1u;
        uint32_t s1 = (first >> (3 * s2)) & 3u, n1 = (first >> (3 * s2 + 2)) & 1u;
        out |= (s1 | ((n1 ^ n2) << 2)) << (3 * o);
    }
    return out;
}

uint32_t perm_inverse(uint32_t code) {
    uint32_t out = 0;
    for (int o = 0; o < 3; ++o) {
        uint32_t s = (code >> (3 * o)) & 3u, ng = (code >> (3 * o + 2)) & 1u;
        out |= (o | (ng << 2)) << (3 * s);
    }
    return out;
}

namespace {

// Gates [i0, i1): STAB_OK, or the error of the first bad gate (its index in *at).
int check_gates(int n, const stab_gate *gates, int64_t i0, int64_t i1, int64_t n_params,
                int64_t *at) {
    for (int64_t i = i0; i < i1; ++i) {
        const stab_gate &g = gates[i];
        *at = i;
        if (g.op > STAB_RZ || g.flags != 0 || g.q0 >= n) return STAB_E_INVAL;
        if (is_two_qubit(g.op) && (g.q1 >= n || g.q1 == g.q0)) return STAB_E_INVAL;
        if (is_rotation(g.op) && (g.param < 0 || g.param >= n_params)) return STAB_E_RANGE;
    }
    return STAB_OK;
}

}  // namespace

int validate_gates(int n, const stab_gate *gates, int64_t m, int64_t n_params, std::string *msg) {
    if (m < 0 || n_params < 0) return STAB_E_RANGE;
    if (m > 0 && gates == nullptr) return STAB_E_INVAL;
    if (m > (int64_t)INT32_MAX / 2) return STAB_E_RANGE;
    // long lists are checked in chunks at once; the first bad gate of the
    // first failing chunk is then described by the walk below
    int64_t from = 0;
    if (m >= kParallelPlanGates) {
        int rc[kPlanChunks];
        int64_t at[kPlanChunks];
        std::vector<std::function<void()>> jobs;
        for (int k = 0; k < kPlanChunks; ++k)
            jobs.push_back([&, k] {
                rc[k] = check_gates(n, gates, m * k / kPlanChunks, m * (k + 1) / kPlanChunks,
                                    n_params, &at[k]);
            });
        HostPool::run(jobs);
        int k = 0;
        while (k < kPlanChunks && rc[k] == STAB_OK) ++k;
        if (k == kPlanChunks) return STAB_OK;
        from = at[k];
    }
    for (int64_t i = from; i < m; ++i) {
        const stab_gate &g = gates[i];
        if (g.op > STAB_RZ || g.flags != 0 || g.q0 >= n) {
            if (msg) *msg = "gate " + std::to_string(i) + ": bad opcode, flags or qubit";
            return STAB_E_INVAL;
        }
        if (is_two_qubit(g.op) && (g.q1 >= n || g.q1 == g.q0)) {
            if (msg) *msg = "gate " + std::to_string(i) + ": bad second qubit";
            return STAB_E_INVAL;
        }
        if (is_rotation(g.op) && (g.param < 0 || g.param >= n_params)) {
            if (msg) *msg = "gate " + std::to_string(i) + ": angle slot out of range";
            return STAB_E_RANGE;
        }
    }
    return STAB_OK;
}

int validate_thetas(const double *thetas, int64_t n_params) {
    if (n_params > 0 && thetas == nullptr) return STAB_E_INVAL;
    for (int64_t j = 0; j < n_params; ++j)
        if (!std::isfinite(thetas[j])) return STAB_E_NONFINITE;
    return STAB_OK;
}

namespace {

struct Emitter {
    HostPlan *P;
    PlanMode mode;
    const std::vector<int32_t> *rot_ordinal;

    void emit_cliff(const stab_gate *gates, int64_t i0, int64_t i1) {
        DevPass p{};
        p.type = P_CLIFF;
        p.first = (uint32_t)P->ops.size();
        for (int64_t i = i0; i < i1; ++i) {
            DevOp op{};
            op.kind = gates[i].op == STAB_CX ? K_CX : K_CZ;
            op.q = gates[i].q0;
            op.q1 = gates[i].q1;
            op.param = -1;
            op.gate = -1;
            P->ops.push_back(op);
        }
        p.n_ops = (uint16_t)(i1 - i0);
        P->passes.push_back(p);
    }

    // One wire's run (gate indices in order) -> one or more P_WIRE passes.
    void emit_wire(const stab_gate *gates, int q, const int64_t *run, size_t run_len) {
        bool as_map = mode == PLAN_ROWS || mode == PLAN_PLAIN_ROWS;
        if (mode == PLAN_FUSED) {
            int n_rot = 0;
            for (size_t k = 0; k < run_len && n_rot <= 3; ++k) n_rot += is_rotation(gates[run[k]].op);
            as_map = n_rot > 3;
        }
        if (as_map) {
            DevMap3 mp{};
            mp.first = (int32_t)P->map_gate_idx.size();
            mp.count = (int32_t)run_len;
            const size_t at = P->map_gate_idx.size();
            P->map_gate_idx.resize(at + run_len);
            for (size_t k = 0; k < run_len; ++k) P->map_gate_idx[at + k] = (int32_t)run[k];
            DevOp op{};
            op.kind = K_MAP3;
            op.q = (uint8_t)q;
            op.param = (int32_t)P->maps.size();
            op.gate = -1;
            P->maps.push_back(mp);
            DevPass p{};
            p.type = P_WIRE;
            p.q = (uint8_t)q;
            p.first = (uint32_t)P->ops.size();
            p.n_ops = 1;
            P->ops.push_back(op);
            P->passes.push_back(p);
            return;
        }
        DevPass p{};
        p.type = P_WIRE;
        p.q = (uint8_t)q;
        p.first = (uint32_t)P->ops.size();
        int rot_in_pass = 0;
        uint32_t pending = kPermIdentity;
        auto flush_perm = [&]() {
            if (pending != kPermIdentity) {
                DevOp op{};
                op.kind = K_PERM;
                op.q = (uint8_t)q;
                op.param = -1;
                op.gate = -1;
                op.perm = (uint16_t)pending;
                op.perm_inv = (uint16_t)perm_inverse(pending);
                P->ops.push_back(op);
            }
            pending = kPermIdentity;
        };
        auto close_pass = [&]() {
            p.n_ops = (uint16_t)(P->ops.size() - p.first);
            if (p.n_ops > 0) P->passes.push_back(p);
            p.first = (uint32_t)P->ops.size();
            rot_in_pass = 0;
        };
        for (size_t k = 0; k < run_len; ++k) {
            const int64_t i = run[k];
            const int op = gates[i].op;
            if (!is_rotation(op)) {
                pending = perm_compose(pending, clifford_perm_code(op));
                if (mode == PLAN_PLAIN) {
                    flush_perm();
                    close_pass();
                }
                continue;
            }
            if (mode == PLAN_GRAD && rot_in_pass == kRotPerGradPass) {
                flush_perm();
                close_pass();
            }
            flush_perm();
            DevOp r{};
            r.kind = K_ROT;
            r.q = (uint8_t)q;
            r.axis = (uint8_t)(op == STAB_RX ? AX_X : op == STAB_RY ? AX_Y : AX_Z);
            r.param = gates[i].param;
            r.gate = (*rot_ordinal)[i];
            P->ops.push_back(r);
            ++rot_in_pass;
            if (mode == PLAN_PLAIN) close_pass();
        }
        flush_perm();
        close_pass();
    }
};

}  // namespace

// Forward conjugation g P g^dagger of one Clifford gate on a string (x, z
// masks), flipping `neg` with the sign: H swaps x and z on the wire (Y -> -Y),
// S: z ^= x (Y -> -X), S^dagger: z ^= x (X -> -Y), X: sign z, Y: sign x ^ z,
// Z: sign x; CX(c, t): x_t ^= x_c, z_c ^= z_t, minus iff x_c z_t (x_t == z_c);
// CZ(a, b): z_a ^= x_b, z_b ^= x_a, minus iff x_a x_b (z_a != z_b).
static void conj_clifford(uint32_t &x, uint32_t &z, uint32_t &neg, uint8_t op, int a, int b) {
    const uint32_t xa = (x >> a) & 1u, za = (z >> a) & 1u;
    const uint32_t ma = 1u << a;
    switch (op) {
    case STAB_H:
        neg ^= xa & za;
        x = (x & ~ma) | (za << a);
        z = (z & ~ma) | (xa << a);
        break;
    case STAB_S: neg ^= xa & za; z ^= xa << a; break;
    case STAB_SDG: neg ^= xa & (za ^ 1u); z ^= xa << a; break;
    case STAB_X: neg ^= za; break;
    case STAB_Y: neg ^= xa ^ za; break;
    case STAB_Z: neg ^= xa; break;
    case STAB_CX: {
        const uint32_t xt = (x >> b) & 1u, zt = (z >> b) & 1u;
        neg ^= xa & zt & ((xt ^ za) ^ 1u);
        x ^= xa << b;
        z ^= zt << a;
        break;
    }
    case STAB_CZ: {
        const uint32_t xb = (x >> b) & 1u, zb = (z >> b) & 1u;
        neg ^= xa & xb & (za ^ zb);
        z ^= xb << a;
        z ^= xa << b;
        break;
    }
    default: break;
    }
}

void clifford_tableau(int n, const stab_gate *gates, int64_t i0, int64_t i1, bool inverse,
                      DevTab *out) {
    std::memset(out, 0, sizeof(*out));
    for (int j = 0; j < 2 * n; ++j) {
        uint32_t x = j < n ? (1u << j) : 0u, z = j < n ? 0u : (1u << (j - n)), neg = 0;
        for (int64_t k = 0; k < i1 - i0; ++k) {
            const stab_gate &g = gates[inverse ? i1 - 1 - k : i0 + k];
            uint8_t op = g.op;
            if (inverse && op == STAB_S) op = STAB_SDG;
            else if (inverse && op == STAB_SDG) op = STAB_S;
            conj_clifford(x, z, neg, op, g.q0, g.q1);
        }
        out->x[j] = x;
        out->z[j] = z;
        out->neg |= (neg & 1u) << j;
    }
}

void build_plan(int n, const stab_gate *gates, int64_t m, int64_t n_params, PlanMode mode,
                HostPlan *out, bool tableaus, bool chunked) {
    HostPlan &P = *out;
    // cleared, not replaced: a context reloading circuits keeps the capacity
    P.passes.clear();
    P.ops.clear();
    P.maps.clear();
    P.map_gate_idx.clear();
    P.param_ptr.clear();
    P.param_rot.clear();
    P.tabs.clear();
    P.n_rot = 0;
    P.n_params = n_params;
    P.mode = mode;
    // the gate list (map composition reads it) and the rotation ordinals
    // (gradient slots, gate order); the slot -> ordinals CSR for gradient plans
    static_assert(sizeof(RawGate) == sizeof(stab_gate) && offsetof(RawGate, param) ==
                      offsetof(stab_gate, param), "RawGate mirrors stab_gate");
    P.raw.resize((size_t)m);
    if (m > 0) std::memcpy(P.raw.data(), gates, (size_t)m * sizeof(RawGate));   // flags are 0
    // (plans that turn every wire run into a map emit no rotation ops and
    // need only the count)
    std::vector<int32_t> &rot_ordinal = P.rot_ordinal;
    int32_t nr = 0;
    if (mode == PLAN_ROWS || mode == PLAN_PLAIN_ROWS) {
        rot_ordinal.clear();
        for (int64_t i = 0; i < m; ++i) nr += is_rotation(gates[i].op);
    } else {
        rot_ordinal.resize((size_t)m);
        for (int64_t i = 0; i < m; ++i) rot_ordinal[i] = is_rotation(gates[i].op) ? nr++ : -1;
    }
    P.n_rot = nr;
    if (mode == PLAN_GRAD) {
        P.param_ptr.assign((size_t)n_params + 1, 0);
        for (int64_t i = 0; i < m; ++i)
            if (rot_ordinal[i] >= 0) P.param_ptr[gates[i].param + 1]++;
        for (int64_t j = 0; j < n_params; ++j) P.param_ptr[j + 1] += P.param_ptr[j];
        P.param_rot.assign((size_t)nr, 0);
        std::vector<int32_t> fill(P.param_ptr.begin(), P.param_ptr.end() - 1);
        for (int64_t i = 0; i < m; ++i)
            if (rot_ordinal[i] >= 0) P.param_rot[fill[gates[i].param]++] = rot_ordinal[i];
    }

    P.passes.reserve((size_t)m + 1);
    P.ops.reserve((size_t)m + 1);
    // Gates [i0, i1) as U_k / V_k passes (Sec. III-A dividing) into `em`;
    // `runs` is scratch (one per concurrent caller).
    auto emit_range_with = [&](Emitter &em, int64_t i0, int64_t i1,
                               std::vector<std::vector<int64_t>> &runs) {
        int64_t i = i0;
        while (i < i1) {
            int64_t j = i;
            if (is_two_qubit(gates[i].op)) {
                while (j < i1 && is_two_qubit(gates[j].op)) ++j;
                if (mode == PLAN_PLAIN || mode == PLAN_PLAIN_ROWS) {
                    for (int64_t k = i; k < j; ++k) em.emit_cliff(gates, k, k + 1);
                } else {
                    // a P_CLIFF pass holds at most 65535 ops
                    for (int64_t k = i; k < j; k += 65535)
                        em.emit_cliff(gates, k, std::min(j, k + 65535));
                }
            } else {
                while (j < i1 && !is_two_qubit(gates[j].op)) ++j;
                if (mode == PLAN_PLAIN || mode == PLAN_PLAIN_ROWS) {
                    for (int64_t k = i; k < j; ++k) em.emit_wire(gates, gates[k].q0, &k, 1);
                } else {
                    for (auto &r : runs) r.clear();
                    for (int64_t k = i; k < j; ++k) runs[gates[k].q0].push_back(k);
                    for (int q = 0; q < n; ++q) {
                        if (runs[q].empty()) continue;
                        // a P_WIRE pass holds at most 65535 ops; cut longer unfused runs
                        const auto &r = runs[q];
                        for (size_t k = 0; k < r.size(); k += 16384)
                            em.emit_wire(gates, q, r.data() + k,
                                         std::min(r.size() - k, (size_t)16384));
                    }
                }
            }
            i = j;
        }
    };
    std::vector<std::vector<int64_t>> runs((size_t)n);
    auto emit_range = [&](Emitter &em, int64_t i0, int64_t i1) {
        emit_range_with(em, i0, i1, runs);
    };
    Emitter em{&P, mode, &rot_ordinal};
    const bool tabs = tableaus && n <= 12 && mode != PLAN_PLAIN && mode != PLAN_PLAIN_ROWS;
    if (!tabs) {
        if (!chunked || m < kParallelPlanGates) {
            emit_range(em, 0, m);
            return;
        }
        // Chunks of the gate list cut where a block of two-qubit gates ends and
        // a block of single-qubit gates begins: the dividing into U_k / V_k is
        // then the same on both sides, so the chunks are planned at once and
        // concatenated (op, map and gate-index references offset).
        std::vector<int64_t> cut = {0};
        for (int w = 1; w < kPlanChunks; ++w) {
            int64_t i = std::max(cut.back() + 1, m * w / kPlanChunks);
            while (i < m && !(is_two_qubit(gates[i - 1].op) && !is_two_qubit(gates[i].op))) ++i;
            if (i < m) cut.push_back(i);
        }
        cut.push_back(m);
        const size_t nc = cut.size() - 1;
        if (nc == 1) {
            emit_range(em, 0, m);
            return;
        }
        std::vector<HostPlan> part(nc);
        std::vector<std::function<void()>> jobs;
        for (size_t k = 0; k < nc; ++k)
            jobs.push_back([&, k] {
                part[k].mode = mode;
                std::vector<std::vector<int64_t>> r((size_t)n);
                Emitter ek{&part[k], mode, &rot_ordinal};
                emit_range_with(ek, cut[k], cut[k + 1], r);
            });
        HostPool::run(jobs);
        size_t np = 0, no = 0, nm = 0, ni = 0;
        std::vector<size_t> op_off(nc), map_off(nc), idx_off(nc), pass_off(nc);
        for (size_t k = 0; k < nc; ++k) {
            pass_off[k] = np;
            op_off[k] = no;
            map_off[k] = nm;
            idx_off[k] = ni;
            np += part[k].passes.size();
            no += part[k].ops.size();
            nm += part[k].maps.size();
            ni += part[k].map_gate_idx.size();
        }
        P.passes.resize(np);
        P.ops.resize(no);
        P.maps.resize(nm);
        P.map_gate_idx.resize(ni);
        jobs.clear();
        for (size_t k = 0; k < nc; ++k)
            jobs.push_back([&, k] {
                const HostPlan &Q = part[k];
                for (size_t i = 0; i < Q.passes.size(); ++i) {
                    DevPass d = Q.passes[i];
                    d.first += (uint32_t)op_off[k];
                    P.passes[pass_off[k] + i] = d;
                }
                for (size_t i = 0; i < Q.ops.size(); ++i) {
                    DevOp o = Q.ops[i];
                    if (o.kind == K_MAP3) o.param += (int32_t)map_off[k];
                    P.ops[op_off[k] + i] = o;
                }
                for (size_t i = 0; i < Q.maps.size(); ++i) {
                    DevMap3 mp = Q.maps[i];
                    mp.first += (int32_t)idx_off[k];
                    P.maps[map_off[k] + i] = mp;
                }
                std::copy(Q.map_gate_idx.begin(), Q.map_gate_idx.end(),
                          P.map_gate_idx.begin() + (ptrdiff_t)idx_off[k]);
            });
        HostPool::run(jobs);
        return;
    }
    // A run of Clifford gates that would take kTabMinPasses or more passes
    // becomes one P_TAB pass: a signed gather through the run's tableau.
    constexpr size_t kTabMinPasses = 4;
    HostPlan scratch;
    scratch.mode = mode;
    int64_t i = 0;
    while (i < m) {
        int64_t j = i;
        while (j < m && !is_rotation(gates[j].op)) ++j;   // Clifford run [i, j)
        if (j - i >= 8) {
            scratch.passes.clear();
            scratch.ops.clear();
            Emitter probe{&scratch, mode, &rot_ordinal};
            emit_range(probe, i, j);
            if (scratch.passes.size() >= kTabMinPasses) {
                DevPass p{};
                p.type = P_TAB;
                p.first = (uint32_t)(P.tabs.size() / 2);
                p.n_ops = 0;
                P.tabs.resize(P.tabs.size() + 2);
                clifford_tableau(n, gates, i, j, true, &P.tabs[P.tabs.size() - 2]);
                clifford_tableau(n, gates, i, j, false, &P.tabs[P.tabs.size() - 1]);
                P.passes.push_back(p);
                i = j;
                continue;
            }
        }
        // the Clifford run (short) and the rotation after it, as usual
        const int64_t e = j < m ? j + 1 : m;
        int64_t k = e;
        // extend over further short runs so ordinary passes still group
        while (k < m) {
            int64_t r = k;
            while (r < m && !is_rotation(gates[r].op)) ++r;
            if (r - k >= 8) break;
            k = r < m ? r + 1 : m;
        }
        emit_range(em, i, k);
        i = k;
    }
}

namespace {

constexpr int kMaxPullPerPass = 64;

// Appends passes to a stream, packing them into chunks of kChunkRecs records
// (a pass never straddles a chunk; an R_NEXT record ends a chunk early).
struct StreamWriter {
    std::vector<Rec> *out;
    std::vector<int32_t> *enc;
    int fill = 0;              // records used in the current chunk
    std::vector<Rec> last;     // the previous pull pass's records, in stream order

    // Header of a pass with n_pull pull records and n_op op records; the
    // caller appends them.
    void header(int q, int n_pull, int n_op) {
        const int need = 1 + n_pull + n_op;
        if (fill + need > kChunkRecs - 1) {
            Rec nx{};
            nx.kind = R_NEXT;
            out->push_back(nx);
            out->resize(out->size() + (kChunkRecs - out->size() % kChunkRecs) % kChunkRecs);
            fill = 0;
        }
        Rec h{};
        h.kind = R_PASS;
        h.q = (uint8_t)q;
        h.param = n_pull;
        h.gate = n_op;
        out->push_back(h);
        fill += need;
    }
    // Pull records [b, e) of the applied two-qubit gates, last applied first;
    // the pass's header (just written) gets kPullRepeat when they equal the
    // previous pull pass's.
    void pulls(const Rec *b, const Rec *e) {
        if (e == b) return;
        const size_t h = out->size() - 1;
        bool same = (size_t)(e - b) == last.size();
        for (size_t k = 0; same && k < last.size(); ++k) {
            const Rec &p = *(e - 1 - k);
            same = p.kind == last[k].kind && p.q == last[k].q && p.q1 == last[k].q1;
        }
        last.clear();
        while (e != b) {
            out->push_back(*--e);
            last.push_back(out->back());
        }
        if (same) (*out)[h].code = kPullRepeat;
    }
    // R_END (the stream ends) or R_NEXT (another piece follows on the next
    // chunk; nothing when the piece is empty), then padding to the chunk end.
    void end(bool last) {
        if (!last && out->empty()) return;
        Rec e{};
        e.kind = last ? R_END : R_NEXT;
        out->push_back(e);
        out->resize(out->size() + (kChunkRecs - out->size() % kChunkRecs) % kChunkRecs);
    }
};

Rec pull_rec(const DevOp &op) {
    Rec r{};
    r.kind = op.kind == K_CX ? R_CX : R_CZ;
    r.q = op.q;
    r.q1 = op.q1;
    return r;
}

}  // namespace

void build_stream(const HostPlan &P, bool backward, std::vector<Rec> *out, int k0, int k1,
                  std::vector<int32_t> *enc, bool last) {
    out->clear();
    if (enc) enc->clear();
    StreamWriter w{out, enc};
    // two-qubit Clifford gates waiting to be pulled, in application order
    std::vector<Rec> applied;
    if (k1 < 0) k1 = (int)P.passes.size();
    const int np = k1 - k0;
    {
        const size_t all = P.passes.size() ? P.passes.size() : 1;
        const size_t share = (size_t)np * (P.ops.size() + P.passes.size()) / all;
        out->reserve(2 * share + (size_t)np + kChunkRecs);
    }
    // The pending pulls: all but the last kMaxPullPerPass-segment go into
    // identity passes; the last goes with the pass on wire q and its ops.
    auto flush_pulls = [&](int q, const DevPass *p) {
        size_t k = 0;
        while (applied.size() - k > (size_t)kMaxPullPerPass) {
            w.header(0, kMaxPullPerPass, 0);
            w.pulls(applied.data() + k, applied.data() + k + kMaxPullPerPass);
            k += kMaxPullPerPass;
        }
        int n_op = 0;
        if (p)
            for (int j = 0; j < p->n_ops; ++j) {
                const int kind = P.ops[p->first + j].kind;
                n_op += (kind == K_ROT || kind == K_PERM) ? 1 : 4;
            }
        w.header(q, (int)(applied.size() - k), n_op);
        w.pulls(applied.data() + k, applied.data() + applied.size());
        applied.clear();
    };
    for (int k = 0; k < np; ++k) {
        const DevPass &p = P.passes[backward ? k1 - 1 - k : k0 + k];
        if (p.type == P_CLIFF) {
            for (int j = 0; j < p.n_ops; ++j) {
                const int jj = backward ? p.n_ops - 1 - j : j;
                applied.push_back(pull_rec(P.ops[p.first + jj]));
            }
            // the gate-by-gate forms keep each two-qubit gate a pass of its own
            if (P.mode == PLAN_PLAIN || P.mode == PLAN_PLAIN_ROWS) flush_pulls(0, nullptr);
            continue;
        }
        flush_pulls(p.q, &p);
        for (int j = 0; j < p.n_ops; ++j) {
            const DevOp &op = P.ops[p.first + (backward ? p.n_ops - 1 - j : j)];
            Rec r{};
            r.q = op.q;
            r.inv = backward ? 1 : 0;
            if (op.kind == K_ROT) {
                r.kind = R_ROT;
                r.axis = op.axis;
                r.param = op.param;
                r.gate = op.gate;
                if (enc) enc->push_back((int32_t)out->size());
                out->push_back(r);
            } else if (op.kind == K_PERM) {
                r.kind = R_PERM;
                r.code = backward ? op.perm_inv : op.perm;
                out->push_back(r);
            } else {
                r.kind = R_MAP3;
                r.param = op.param;
                if (enc) enc->push_back((int32_t)out->size());
                out->push_back(r);
                Rec d{};
                d.kind = R_DATA;
                out->push_back(d);
                out->push_back(d);
                out->push_back(d);
            }
        }
    }
    if (!applied.empty()) flush_pulls(0, nullptr);
    w.end(last);
}

int encode_terms(int n, const stab_term *O, int64_t n_terms, std::vector<DevTerm> *out) {
    out->clear();
    if (n_terms < 0) return STAB_E_RANGE;
    if (n_terms > 0 && O == nullptr) return STAB_E_INVAL;
    const uint64_t lim = 1ull << n;
    std::map<uint64_t, double> acc;
    for (int64_t k = 0; k < n_terms; ++k) {
        if (O[k].x >= lim || O[k].z >= lim) return STAB_E_INVAL;
        if (!std::isfinite(O[k].coeff)) return STAB_E_NONFINITE;
        acc[O[k].z | (O[k].x << n)] += O[k].coeff;
    }
    for (auto &kv : acc) out->push_back(DevTerm{kv.second, kv.first});
    return STAB_OK;
}

}  // namespace stab
