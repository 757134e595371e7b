"""Pins of the sparse-list oracle (term lists of (coefficient, string), n <= 32).

It is pinned to things other than itself: the dense oracle (an independent
restatement of Table I and the map_CX list) bit for bit at small n, a CHP
stabilizer tableau for Clifford circuits up to n = 32, closed forms of product
and GHZ circuits at n = 30, a state-vector simulation, and invariants.  Planted
mistakes in copies of its source must fail these pins.
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import chp_ref
import dense_ref as D
import oracle
from paper_2502_10685_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "sparse_oracle.c")


def as_dense(n, keys, vals):
    d = np.zeros(4 ** n)
    d[np.asarray(keys, dtype=np.int64)] = vals
    return d


def key_of(s):
    k = 0
    for ch in s:
        k = k * 4 + "IXYZ".index(ch)
    return k


# ---------------------------------------------------------------- vs the dense oracle

@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_generators_equal_dense_oracle_bitwise(n):
    for seed in range(4):
        c = W.random_circuit(n, 150, seed=300 + 10 * n + seed)
        G = oracle.generators(n, c.gates, c.thetas)
        for k in range(n):
            keys, vals = oracle.sparse_generator(n, c.gates, c.thetas, k)
            assert np.all(np.diff(keys.astype(np.float64)) > 0)     # sorted, unique
            assert np.all(vals != 0.0)
            np.testing.assert_array_equal(as_dense(n, keys, vals), G[k])


@pytest.mark.parametrize("n", [2, 4, 5])
def test_backward_observables_equal_dense_oracle(n):
    for seed in range(3):
        c = W.random_circuit(n, 120, seed=500 + 10 * n + seed)
        obs = W.random_observable(n, 6, seed=seed)
        keys, vals = oracle.sparse_terms(n, obs)
        k2, v2 = oracle.sparse_propagate(n, c.gates, c.thetas, keys, vals, backward=True)
        want = oracle.backward(n, c.gates, c.thetas, oracle.dense_observable(n, obs))
        np.testing.assert_array_equal(as_dense(n, k2, v2), want)
        assert oracle.sparse_expect(n, c.gates, c.thetas, obs) == pytest.approx(
            oracle.expect(n, c.gates, c.thetas, obs), abs=1e-14)


def test_statevector_expectations_n7():
    n = 7
    for seed in range(3):
        c = W.random_circuit(n, 80, seed=600 + seed)
        obs = W.random_observable(n, 5, seed=seed) + [(0.3, "Z" * n)]
        got = oracle.sparse_expect(n, c.gates, c.thetas, obs)
        want = D.statevector_expect(n, c.gates, c.thetas, obs)
        assert abs(got - want) <= 1e-12


# ---------------------------------------------------------------- large n

@pytest.mark.parametrize("n", [12, 20, 32])
def test_clifford_circuits_match_chp_tableau_large_n(n):
    rng = np.random.default_rng(70 + n)
    items = []
    for _ in range(20 * n):
        kind = int(rng.integers(3))
        a = int(rng.integers(n))
        if kind == 0:
            items.append(("H", a))
        elif kind == 1:
            items.append(("S", a))
        else:
            b = int((a + 1 + rng.integers(n - 1)) % n)
            items.append(("CX", a, b))
    gates = W.gates_from_list(items)
    tab = chp_ref.Tableau(n)
    for it in items:
        if it[0] == "H":
            tab.h(it[1])
        elif it[0] == "S":
            tab.s(it[1])
        else:
            tab.cnot(it[1], it[2])
    for k in range(n):
        keys, vals = oracle.sparse_generator(n, gates, np.zeros(0), k)
        sign, s = tab.row(k)
        assert keys.tolist() == [key_of(s)]
        assert vals.tolist() == [float(sign)]


def test_product_rotations_closed_form_n30():
    """RX(theta_q) on every qubit: <Z_q> = cos theta_q, <Z_a Z_b> = cos cos,
    <Z_0..Z_11> = prod cos, <Y_q> = -sin theta_q."""
    n = 30
    rng = np.random.default_rng(3)
    th = rng.uniform(0, 2 * math.pi, size=n)
    gates = W.gates_from_list([("RX", q, j) for j, q in enumerate(range(n))])
    for q in (0, 13, 29):
        s = "I" * q + "Z" + "I" * (n - q - 1)
        assert oracle.sparse_expect(n, gates, th, [(1.0, s)]) == pytest.approx(
            math.cos(th[q]), abs=1e-15)
        y = "I" * q + "Y" + "I" * (n - q - 1)
        assert oracle.sparse_expect(n, gates, th, [(1.0, y)]) == pytest.approx(
            -math.sin(th[q]), abs=1e-15)
    zz = ["I"] * n
    zz[4] = zz[22] = "Z"
    assert oracle.sparse_expect(n, gates, th, [(1.0, "".join(zz))]) == pytest.approx(
        math.cos(th[4]) * math.cos(th[22]), abs=1e-15)
    # Z on the first 12 qubits: the backward list doubles per rotation it meets
    z12 = "Z" * 12 + "I" * (n - 12)
    assert oracle.sparse_expect(n, gates, th, [(1.0, z12)]) == pytest.approx(
        float(np.prod(np.cos(th[:12]))), abs=1e-15)


def test_ghz_phase_closed_form_n30():
    """H, a CX chain and RZ(phi) on one qubit: <X...X> = cos(phi), <Z_0 Z_k> = 1."""
    n = 30
    for phi, q in ((0.37, 0), (2.9, 17)):
        items = [("H", 0)] + [("CX", k, k + 1) for k in range(n - 1)] + [("RZ", q, 0)]
        gates = W.gates_from_list(items)
        th = np.array([phi])
        assert oracle.sparse_expect(n, gates, th, [(1.0, "X" * n)]) == pytest.approx(
            math.cos(phi), abs=1e-14)
        zz = "Z" + "I" * (n - 2) + "Z"
        assert oracle.sparse_expect(n, gates, th, [(1.0, zz)]) == pytest.approx(1.0, abs=1e-15)


def test_generator_norm_and_identity_free_n24():
    """Conjugation keeps sum lambda^2 = 1 and never creates the identity term."""
    n = 24
    c = W.clifford_plus_rotations(n, 400, 14, seed=8)
    for k in (0, 11, 23):
        keys, vals = oracle.sparse_generator(n, c.gates, c.thetas, k)
        assert abs(float(np.sum(vals * vals)) - 1.0) <= 1e-12
        assert 0 not in keys.tolist()


def test_forward_then_backward_is_identity_n16():
    n = 16
    c = W.clifford_plus_rotations(n, 300, 12, seed=12)
    keys, vals = oracle.sparse_terms(n, [(0.7, "XZ" + "I" * (n - 3) + "Y"), (-0.2, "Z" * n)])
    k1, v1 = oracle.sparse_propagate(n, c.gates, c.thetas, keys, vals)
    k2, v2 = oracle.sparse_propagate(n, c.gates, c.thetas, k1, v1, backward=True)
    got = dict(zip(k2.tolist(), v2.tolist()))
    want = dict(zip(keys.tolist(), vals.tolist()))
    for k in set(got) | set(want):
        assert abs(got.get(k, 0.0) - want.get(k, 0.0)) <= 1e-12


def test_overflow_reported():
    n = 10
    c = W.layered_ansatz(n, 40, seed=2)
    with pytest.raises(OverflowError):
        oracle.sparse_propagate(n, c.gates, c.thetas, *oracle.sparse_terms(n, [(1.0, "Z" * n)]),
                                cap=16)


# ---------------------------------------------------------------- planted mistakes

MUTATIONS = {
    "rx_sign": ("o[2] = w[2] * c - w[3] * s;", "o[2] = w[2] * c + w[3] * s;"),
    "cx_sign": ('{"XZ", "-YY"}', '{"XZ", "YY"}'),
    "letter_order": ("return (int)((key >> (2 * (n - 1 - q))) & 3u);",
                     "return (int)((key >> (2 * q)) & 3u);"),
    "merge_keeps_first": ("while (j < t->len && tmp[j].k == tmp[i].k) acc += tmp[j++].v;",
                          "acc = tmp[i].v; while (j < t->len && tmp[j].k == tmp[i].k) j++;"),
    "inverse_rotation": ("case SP_RZ: rc = apply_row(t, n, q, ROW_RZ, c, inverse ? -s : s);",
                         "case SP_RZ: rc = apply_row(t, n, q, ROW_RZ, c, s);"),
}


def _mutant(name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert old in src, name
    src = src.replace(old, new, 1)
    d = tempfile.mkdtemp(prefix="sparsemut_")
    path = os.path.join(d, "m.c")
    with open(path, "w") as f:
        f.write(src)
    so = os.path.join(d, "m.so")
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, path,
                           "-lm"])
    L = ctypes.CDLL(so)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.orc_sparse_expect.argtypes = [ctypes.c_int, i64, vp, vp, i64, i64, vp, vp, vp]
    return L


def _pins_fail(L):
    """True when any of a few pins rejects the library L."""
    checks = []
    for n, seed in ((3, 1), (4, 2), (5, 3)):
        c = W.random_circuit(n, 120, seed=900 + seed)
        obs = W.random_observable(n, 4, seed=seed)
        keys, vals = oracle.sparse_terms(n, obs)
        out = ctypes.c_double()
        th = np.ascontiguousarray(c.thetas if c.thetas.size else np.zeros(1))
        L.orc_sparse_expect(n, c.m, c.gates.ctypes.data, th.ctypes.data, c.n_params, keys.size,
                            keys.ctypes.data, vals.ctypes.data, ctypes.byref(out))
        checks.append(abs(out.value - D.statevector_expect(n, c.gates, c.thetas, obs)))
    return max(checks) > 1e-6


def test_unmutated_sparse_oracle_passes():
    L = ctypes.CDLL(oracle.build())
    L.orc_sparse_expect.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert not _pins_fail(L)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    assert _pins_fail(_mutant(name))
