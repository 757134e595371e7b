"""Seeded synthetic inputs: gate lists, angles, observables, batches, traces.

This module only draws random circuits in the public gate-record format; it
holds none of the propagation arithmetic, so both the CUDA library and the CPU
oracle can be fed from it.

Gate record (8 bytes, the layout of ``stab_gate`` in the C interface)::

    op:u8  q0:u8  q1:u8  flags:u8  param:i32

``op`` numbers the gates H, S, Sdg, X, Y, Z, CX, CZ, RX, RY, RZ as 0..10; for
CX ``q0`` is the control and ``q1`` the target; rotations read their angle
from ``thetas[param]`` (the paper's instruction tuple {g, w, theta}, Sec. III-A,
with the angle moved to a parameter slot so that many gates can share one
trainable value); Clifford gates carry ``param = -1``.

Observables are lists of ``(coeff, string)`` with one letter per qubit,
qubit 0 first, e.g. ``[(1.0, "ZZII")]``.

Workload shapes follow the paper's W_chain + ZXZ experiments (Sec. V) and the
layered ansatz with a CNOT ring; every draw is seeded (numpy PCG64).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

OPS = {"H": 0, "S": 1, "SDG": 2, "X": 3, "Y": 4, "Z": 5, "CX": 6, "CZ": 7,
       "RX": 8, "RY": 9, "RZ": 10}
OP_NAMES = {v: k for k, v in OPS.items()}
TWO_QUBIT = (OPS["CX"], OPS["CZ"])
ROTATIONS = (OPS["RX"], OPS["RY"], OPS["RZ"])

GATE_DTYPE = np.dtype([("op", "u1"), ("q0", "u1"), ("q1", "u1"), ("flags", "u1"),
                       ("param", "<i4")])
assert GATE_DTYPE.itemsize == 8

Observable = List[Tuple[float, str]]


@dataclasses.dataclass
class Circuit:
    """A gate list over ``n`` qubits with its parameter vector."""
    n: int
    gates: np.ndarray          # GATE_DTYPE records, length m
    thetas: np.ndarray         # float64, length n_params

    @property
    def m(self) -> int:
        return int(self.gates.shape[0])

    @property
    def n_params(self) -> int:
        return int(self.thetas.shape[0])

    def with_thetas(self, thetas: np.ndarray) -> "Circuit":
        return Circuit(self.n, self.gates, np.ascontiguousarray(thetas, dtype=np.float64))


def gates_from_list(items: Sequence[Tuple]) -> np.ndarray:
    """``[("H", 0), ("CX", 0, 1), ("RX", 2, slot), ...]`` -> record array.

    Rotations take ``(name, qubit, slot)``; two-qubit gates ``(name, q0, q1)``.
    """
    out = np.zeros(len(items), dtype=GATE_DTYPE)
    for i, it in enumerate(items):
        op = OPS[it[0]]
        out[i]["op"] = op
        out[i]["q0"] = it[1]
        out[i]["param"] = -1
        if op in TWO_QUBIT:
            out[i]["q1"] = it[2]
        elif op in ROTATIONS:
            out[i]["param"] = it[2]
    return out


def layered_ansatz(n: int, m: int, seed: int, p_replace: float = 0.1) -> Circuit:
    """Repeated layers of RX, RY, RZ on every qubit, then a CNOT ring.

    Per qubit q = 0..n-1 the layer has the slots RX(q), RY(q), RZ(q); each slot
    is independently replaced, with probability ``p_replace``, by H or S
    (50/50).  The ring is CX(q -> q+1 mod n) for q = 0..n-1 (none for n = 1).
    Every surviving rotation gets its own slot with theta ~ U[0, 2 pi).  The
    list is cut at exactly ``m`` gates, so the last layer may be partial.
    Draws (PCG64): one uniform per rotation slot for the replacement test, one
    for the H/S choice and one angle, each as an array over all slots.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ring = n if n >= 2 else 0
    per_layer = 3 * n + ring
    layers = -(-m // per_layer) if m > 0 else 0
    # one layer's template
    t_op = np.empty(per_layer, dtype=np.uint8)
    t_q0 = np.empty(per_layer, dtype=np.uint8)
    t_q1 = np.zeros(per_layer, dtype=np.uint8)
    rot = np.zeros(per_layer, dtype=bool)
    k = 0
    for q in range(n):
        for r in ("RX", "RY", "RZ"):
            t_op[k], t_q0[k], rot[k] = OPS[r], q, True
            k += 1
    for q in range(ring):
        t_op[k], t_q0[k], t_q1[k] = OPS["CX"], q, (q + 1) % n
        k += 1
    op = np.tile(t_op, layers)[:m]
    q0 = np.tile(t_q0, layers)[:m]
    q1 = np.tile(t_q1, layers)[:m]
    is_rot = np.tile(rot, layers)[:m]
    n_slots = int(is_rot.sum())
    u = rng.random(n_slots)
    hs = rng.random(n_slots) < 0.5
    theta = rng.uniform(0.0, 2.0 * math.pi, n_slots)
    replaced = u < p_replace
    slot_ops = op[is_rot].copy()
    slot_ops[replaced] = np.where(hs[replaced], OPS["H"], OPS["S"])
    op[is_rot] = slot_ops
    param = np.full(m, -1, dtype=np.int32)
    keep = ~replaced
    slot_param = np.full(n_slots, -1, dtype=np.int32)
    slot_param[keep] = np.arange(int(keep.sum()), dtype=np.int32)
    param[is_rot] = slot_param
    recs = np.zeros(m, dtype=GATE_DTYPE)
    recs["op"], recs["q0"], recs["q1"], recs["param"] = op, q0, q1, param
    return Circuit(n, recs, np.ascontiguousarray(theta[keep], dtype=np.float64))


def paper_shaped_ansatz(n: int, layers: int, repeats: int, seed: int) -> Circuit:
    """W_chain + ZXZ shape of Sec. V: per layer a CNOT ring, then ``repeats``
    blocks of RZ, RX, RZ on every qubit (n=4, 50 layers, 100 repeats gives
    50 x (4 + 1200) = 60,200 gates)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    items = []
    thetas: List[float] = []
    ring = [(q, (q + 1) % n) for q in range(n)] if n >= 2 else []
    for _ in range(layers):
        for (c, t) in ring:
            items.append(("CX", c, t))
        for _ in range(repeats):
            for q in range(n):
                for rot in ("RZ", "RX", "RZ"):
                    items.append((rot, q, len(thetas)))
                    thetas.append(rng.uniform(0.0, 2.0 * math.pi))
    return Circuit(n, gates_from_list(items), np.asarray(thetas, dtype=np.float64))


def random_circuit(n: int, m: int, seed: int, clifford_only: bool = False,
                   ops: Sequence[str] | None = None, shared_params: int = 0) -> Circuit:
    """Uniformly mixed gates over every opcode (or ``ops``), for parity tests.

    With ``shared_params > 0`` rotations draw their slot from that many shared
    parameters, so a slot can be read by several gates.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if ops is None:
        ops = ["H", "S", "SDG", "X", "Y", "Z", "CX", "CZ"]
        if not clifford_only:
            ops = ops + ["RX", "RY", "RZ"] * 2
    if n < 2:
        ops = [o for o in ops if OPS[o] not in TWO_QUBIT]
    recs = np.zeros(m, dtype=GATE_DTYPE)
    thetas: List[float] = []
    if shared_params > 0:
        thetas = list(rng.uniform(0.0, 2.0 * math.pi, size=shared_params))
    for i in range(m):
        op = OPS[ops[int(rng.integers(len(ops)))]]
        q0 = int(rng.integers(n))
        q1 = 0
        param = -1
        if op in TWO_QUBIT:
            q1 = int(rng.integers(n - 1))
            if q1 >= q0:
                q1 += 1
        elif op in ROTATIONS:
            if shared_params > 0:
                param = int(rng.integers(shared_params))
            else:
                param = len(thetas)
                thetas.append(rng.uniform(0.0, 2.0 * math.pi))
        recs[i] = (op, q0, q1, 0, param)
    return Circuit(n, recs, np.asarray(thetas, dtype=np.float64))



def clifford_plus_rotations(n: int, m: int, n_rot: int, seed: int,
                            two_qubit_fraction: float = 0.4) -> Circuit:
    """``m`` gates: random Clifford gates (H, S, S^dagger, X, Y, Z, CX, CZ) with
    ``n_rot`` rotations (R_x, R_y, R_z, own slot each, theta ~ U[0, 2 pi)) at
    random positions.  The stabilizer order of a generator grows at most by
    a factor 2 per rotation (Sec. II-B), so these circuits stay sparse for
    any n; they are the workload of the sparse representation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_rot = min(n_rot, m)
    rot_at = set(int(i) for i in rng.choice(m, size=n_rot, replace=False)) if n_rot else set()
    one_q = ["H", "S", "SDG", "X", "Y", "Z"]
    recs = np.zeros(m, dtype=GATE_DTYPE)
    thetas: List[float] = []
    for i in range(m):
        q0 = int(rng.integers(n))
        q1, param = 0, -1
        if i in rot_at:
            op = OPS[("RX", "RY", "RZ")[int(rng.integers(3))]]
            param = len(thetas)
            thetas.append(rng.uniform(0.0, 2.0 * math.pi))
        elif n > 1 and rng.uniform() < two_qubit_fraction:
            op = OPS["CX"] if rng.uniform() < 0.75 else OPS["CZ"]
            q1 = int(rng.integers(n - 1))
            if q1 >= q0:
                q1 += 1
        else:
            op = OPS[one_q[int(rng.integers(len(one_q)))]]
        recs[i] = (op, q0, q1, 0, param)
    return Circuit(n, recs, np.asarray(thetas, dtype=np.float64))

# ---------------------------------------------------------------- observables

def obs_z(n: int, k: int) -> Observable:
    """Z on qubit k."""
    s = ["I"] * n
    s[k] = "Z"
    return [(1.0, "".join(s))]


def obs_zz(n: int, a: int, b: int) -> Observable:
    s = ["I"] * n
    s[a] = "Z"
    s[b] = "Z"
    return [(1.0, "".join(s))]


def obs_chain(n: int, periodic: bool = False, x_weight: float = 0.5) -> Observable:
    """sum_i Z_i Z_{i+1} + x_weight * sum_i X_i (open chain unless periodic)."""
    terms: Observable = []
    last = n if periodic else n - 1
    for i in range(last):
        s = ["I"] * n
        s[i] = "Z"
        s[(i + 1) % n] = "Z"
        terms.append((1.0, "".join(s)))
    for i in range(n):
        s = ["I"] * n
        s[i] = "X"
        terms.append((x_weight, "".join(s)))
    return terms


def random_observable(n: int, n_terms: int, seed: int) -> Observable:
    rng = np.random.Generator(np.random.PCG64(seed))
    out: Observable = []
    for _ in range(n_terms):
        s = "".join("IXYZ"[int(rng.integers(4))] for _ in range(n))
        out.append((float(rng.normal()), s))
    return out


# ---------------------------------------------------------------- batches

@dataclasses.dataclass
class BatchItem:
    circuit: Circuit
    kind: str                 # "generators" or "expect"
    observable: Observable | None = None


def psr_variants(circ: Circuit) -> List[Circuit]:
    """All 2m parameter-shift copies (theta_j +- pi/2) of ``circ`` (Sec. I)."""
    out = []
    for j in range(circ.n_params):
        for sgn in (1.0, -1.0):
            th = circ.thetas.copy()
            th[j] += sgn * math.pi / 2
            out.append(circ.with_thetas(th))
    return out


def uneven_batch(n_circuits: int, seed: int, n_range=(2, 8), depth_range=(100, 20000),
                 psr_base: Tuple[int, int] | None = (6, 2000),
                 psr_observable: Observable | None = None) -> List[BatchItem]:
    """Uneven batch: the 2m parameter-shift variants of a layered ansatz of
    ``psr_base = (n, depth)`` (expectation units), then random layered
    circuits with n ~ U{n_range} and depth ~ U[depth_range] (generator units),
    ``n_circuits`` items in total."""
    rng = np.random.Generator(np.random.PCG64(seed))
    items: List[BatchItem] = []
    if psr_base is not None:
        pn, pd = psr_base
        base = layered_ansatz(pn, pd, seed + 7)
        obs = psr_observable if psr_observable is not None else obs_chain(pn)
        for v in psr_variants(base)[:n_circuits]:
            items.append(BatchItem(v, "expect", obs))
    k = 0
    while len(items) < n_circuits:
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        d = int(rng.integers(depth_range[0], depth_range[1] + 1))
        items.append(BatchItem(layered_ansatz(n, d, seed + 1000 + k), "generators"))
        k += 1
    return items


@dataclasses.dataclass
class Request:
    arrival_s: float
    circuit: Circuit
    kind: str                 # "expect" or "grad"
    observable: Observable


def serving_trace(n_requests: int, seed: int, rate_per_s: float = 2000.0,
                  n_range=(4, 12), depth_range=(100, 60000)) -> List[Request]:
    """Poisson arrivals; n ~ U{n_range}; depth log-uniform in depth_range;
    50/50 expectation / gradient requests on the chain observable."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out: List[Request] = []
    lo, hi = math.log(depth_range[0]), math.log(depth_range[1])
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate_per_s))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        d = int(round(math.exp(rng.uniform(lo, hi))))
        kind = "expect" if rng.random() < 0.5 else "grad"
        out.append(Request(t, layered_ansatz(n, d, seed * 100003 + i), kind, obs_chain(n)))
    return out
