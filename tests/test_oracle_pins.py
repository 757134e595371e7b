"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
worked examples and tables (tests/golden/paper_examples.json), dense 2^n
matrices, a stabilizer tableau, a state-vector simulation, invariants and
closed forms.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2502_10685_gb300 import workloads as W

import chp_ref
import dense_ref as D

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))
OPS = W.OPS


def idx(s):
    return oracle.string_to_index(s)


# ---------------------------------------------------------------- paper examples

def test_example2_string_index():
    e = GOLD["example2"]
    assert oracle.string_to_index(e["string"]) == e["index"]
    assert oracle.index_to_string(3, e["index"]) == e["string"]
    # extremes stated in Sec. III-B: I..I -> 0, Z..Z -> 4^n - 1
    assert oracle.string_to_index("IIII") == 0
    assert oracle.string_to_index("ZZZZ") == 4 ** 4 - 1


def test_example1_two_rotations():
    e = GOLD["example1"]
    rng = np.random.default_rng(11)
    for _ in range(5):
        t1, t2 = rng.uniform(0, 2 * math.pi, size=2)
        gates = W.gates_from_list([("RY", 0, 0), ("RX", 0, 1)])
        v0 = np.zeros(4)
        v0[idx(e["initial"])] = 1.0
        env = {"theta1": t1, "theta2": t2, "cos": math.cos, "sin": math.sin}
        v1 = oracle.forward(1, gates[:1], np.array([t1, t2]), v0)
        exp1 = np.zeros(4)
        for s, f in e["after_first"].items():
            exp1[idx(s)] = eval(f, {}, env)
        np.testing.assert_allclose(v1, exp1, atol=1e-15)
        v2 = oracle.forward(1, gates, np.array([t1, t2]), v0)
        exp2 = np.zeros(4)
        for s, f in e["after_second"].items():
            exp2[idx(s)] = eval(f, {}, env)
        np.testing.assert_allclose(v2, exp2, atol=1e-15)


def test_example3_encode_expand():
    e = GOLD["example3"]
    out = oracle.expand(np.array(e["encoded"], dtype=float))
    np.testing.assert_array_equal(out[: len(e["printed_prefix"])], e["printed_prefix"])
    nz = sorted(np.nonzero(out)[0].tolist())
    assert nz == sorted(idx(s) for s in e["nonzero_strings"])
    assert np.all(out[nz] == 1.0)


def test_example4_flatten_reduce():
    e = GOLD["example4"]
    W4 = np.array(e["encoded"], dtype=float)
    row = oracle.expand(W4[:1])
    for k, v in e["printed_row_entries"].items():
        assert row[int(k)] == v
    red = oracle.expand(W4)
    for k, v in e["printed_reduce_entries"].items():
        assert red[int(k)] == v
    np.testing.assert_array_equal(red, 2 * row)
    # Kronecker reading of the elided middle: row = kron([1,2,3,4],[1,2,3,4])
    np.testing.assert_array_equal(row, np.kron([1, 2, 3, 4], [1, 2, 3, 4]))


def test_table1_rows_as_printed():
    t = GOLD["table1"]
    rng = np.random.default_rng(3)
    for name, row in t.items():
        if name.startswith("_"):
            continue
        for _ in range(4):
            w = rng.normal(size=4)
            th = rng.uniform(0, 2 * math.pi)
            c, s = math.cos(th), math.sin(th)
            env = {"w0": w[0], "w1": w[1], "w2": w[2], "w3": w[3], "c": c, "s": s}
            expected = [eval(ex, {}, env) for ex in row]
            got = oracle.map_noncx(OPS[name], w, c, s)
            np.testing.assert_allclose(got, expected, rtol=0, atol=1e-15)


def test_cx_rule_list_as_printed():
    r = GOLD["cx_rules"]
    g = W.gates_from_list([("CX", 0, 1)])

    def image(s):
        v = np.zeros(16)
        v[idx(s)] = 1.0
        out = oracle.forward(2, g, np.zeros(1), v)
        (nz,) = np.nonzero(out)
        assert len(nz) == 1
        return out[nz[0]], oracle.index_to_string(2, nz[0])

    seen = set()
    for a, b in r["swap"]:
        assert image(a) == (1.0, b) and image(b) == (1.0, a)
        seen |= {a, b}
    for a in r["fixed"]:
        assert image(a) == (1.0, a)
        seen.add(a)
    for a, b in r["swap_negated"]:
        assert image(a) == (-1.0, b) and image(b) == (-1.0, a)
        seen |= {a, b}
    assert len(seen) == 16


# ---------------------------------------------------------------- dense matrices

ALL_GATES = ["H", "S", "SDG", "X", "Y", "Z", "CX", "CZ", "RX", "RY", "RZ"]


@pytest.mark.parametrize("name", ALL_GATES)
@pytest.mark.parametrize("n", [2, 3])
def test_every_gate_against_dense_conjugation(name, n):
    """c'_P = Tr(P G A G^dagger) / 2^n for A = sum_P v_P P, forward and inverse."""
    rng = np.random.default_rng(100 + n)
    op = OPS[name]
    for trial in range(3):
        q0 = int(rng.integers(n))
        q1 = int((q0 + 1 + rng.integers(n - 1)) % n)
        th = float(rng.uniform(0, 2 * math.pi))
        v = rng.normal(size=4 ** n)
        G = D.gate_matrix(n, op, q0, q1, th)
        A = D.coeffs_to_matrix(n, v)
        want_fwd = D.matrix_to_coeffs(n, G @ A @ G.conj().T)
        want_inv = D.matrix_to_coeffs(n, G.conj().T @ A @ G)
        got_fwd = oracle.apply_gate(n, op, q0, q1, v, math.cos(th), math.sin(th), False)
        got_inv = oracle.apply_gate(n, op, q0, q1, v, math.cos(th), math.sin(th), True)
        np.testing.assert_allclose(got_fwd, want_fwd, atol=1e-12)
        np.testing.assert_allclose(got_inv, want_inv, atol=1e-12)


def test_generators_brute_force_n3():
    """c_P(U Z_k U^dagger) = Tr(P U Z_k U^dagger) / 2^n for a random circuit."""
    n = 3
    c = W.random_circuit(n, 40, seed=5)
    U = D.circuit_unitary(n, c.gates, c.thetas)
    got = oracle.generators(n, c.gates, c.thetas)
    for k in range(n):
        Zk = D.pauli_matrix("".join("Z" if q == k else "I" for q in range(n)))
        want = D.matrix_to_coeffs(n, U @ Zk @ U.conj().T)
        np.testing.assert_allclose(got[k], want, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_expectation_against_statevector(n):
    for seed in range(2):
        c = W.random_circuit(n, 30 * n, seed=200 + 10 * n + seed)
        obs = W.random_observable(n, 5, seed=300 + n + seed)
        got = oracle.expect(n, c.gates, c.thetas, obs)
        want = D.statevector_expect(n, c.gates, c.thetas, obs)
        assert abs(got - want) <= 1e-12 * sum(abs(a) for a, _ in obs)


def test_layered_ansatz_expectation_against_statevector():
    n = 5
    c = W.layered_ansatz(n, 400, seed=1001)
    obs = W.obs_chain(n)
    got = oracle.expect(n, c.gates, c.thetas, obs)
    want = D.statevector_expect(n, c.gates, c.thetas, obs)
    assert abs(got - want) <= 1e-12 * sum(abs(a) for a, _ in obs)


# ---------------------------------------------------------------- tableau

@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_clifford_circuits_match_chp_tableau(n):
    rng = np.random.default_rng(40 + n)
    items = []
    for _ in range(60 * n):
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
    gens = oracle.generators(n, gates, np.zeros(0))
    for k in range(n):
        sign, s = tab.row(k)
        want = np.zeros(4 ** n)
        want[idx(s)] = sign
        # bit-exact: a single +-1 entry, zeros elsewhere
        np.testing.assert_array_equal(gens[k], want)


def test_clifford_all_opcodes_single_strings():
    """Every Clifford opcode keeps each generator a single +-1 string (bit-exact)."""
    for n in (2, 4, 6):
        c = W.random_circuit(n, 300, seed=77 + n, clifford_only=True)
        gens = oracle.generators(n, c.gates, c.thetas)
        for k in range(n):
            nz = np.nonzero(gens[k])[0]
            assert len(nz) == 1 and abs(gens[k][nz[0]]) == 1.0


# ---------------------------------------------------------------- invariants

def test_norm_conserved_every_gate():
    n = 4
    c = W.random_circuit(n, 400, seed=9)
    v = oracle.generator(n, 2)
    for i in range(c.m):
        v = oracle.forward(n, c.gates[i:i + 1], c.thetas, v)
        assert abs(np.dot(v, v) - 1.0) < 1e-13
        assert v[0] == 0.0   # identity coefficient of a generator stays 0


def test_norm_drift_deep_circuit():
    n = 4
    c = W.layered_ansatz(n, 60200, seed=1002)
    gens = oracle.generators(n, c.gates, c.thetas)
    for k in range(n):
        assert abs(np.dot(gens[k], gens[k]) - 1.0) < 1e-12


def test_rho_purity_and_trace_with_generators():
    """r = forward-evolved indicator of {I,Z}^n (2^n rho in the Pauli basis):
    sum r_P^2 = 2^n (purity), r_I = 1, and Tr(rho S_k) = sum_P r_P c_P(S_k) = 1."""
    n = 4
    c = W.layered_ansatz(n, 500, seed=21)
    r0 = np.zeros(4 ** n)
    for i in range(4 ** n):
        if all(ch in "IZ" for ch in oracle.index_to_string(n, i)):
            r0[i] = 1.0
    r = oracle.forward(n, c.gates, c.thetas, r0)
    assert abs(np.dot(r, r) - 2 ** n) < 1e-10
    assert abs(r[0] - 1.0) < 1e-13
    gens = oracle.generators(n, c.gates, c.thetas)
    for k in range(n):
        assert abs(np.dot(r, gens[k]) - 1.0) < 1e-12


def test_duality_forward_backward():
    """c_Q(U^dagger P U) = c_P(U Q U^dagger)."""
    n = 4
    c = W.random_circuit(n, 200, seed=31)
    gens = oracle.generators(n, c.gates, c.thetas)
    for k in range(n):
        for s in ("ZZII", "XIYZ", "IYYI"):
            O = oracle.dense_observable(n, [(1.0, s)])
            back = oracle.backward(n, c.gates, c.thetas, O)
            zk = "".join("Z" if q == k else "I" for q in range(n))
            assert abs(back[idx(zk)] - gens[k][idx(s)]) < 1e-13


# ---------------------------------------------------------------- closed forms

def test_theta_zero_is_identity():
    n = 3
    rng = np.random.default_rng(1)
    v = rng.normal(size=4 ** n)
    for name in ("RX", "RY", "RZ"):
        for q in range(n):
            out = oracle.apply_gate(n, OPS[name], q, 0, v, 1.0, 0.0)
            np.testing.assert_array_equal(out, v)
            g = W.gates_from_list([(name, q, 0)])
            out2 = oracle.forward(n, g, np.array([0.0]), v)
            np.testing.assert_array_equal(out2, v)


def test_rz_half_pi_is_s_and_pi_rotations_are_paulis():
    n = 2
    rng = np.random.default_rng(2)
    v = rng.normal(size=16)
    for q in range(n):
        s_gate = oracle.apply_gate(n, OPS["S"], q, 0, v)
        rz_exact = oracle.apply_gate(n, OPS["RZ"], q, 0, v, 0.0, 1.0)
        np.testing.assert_array_equal(rz_exact, s_gate)
        g = W.gates_from_list([("RZ", q, 0)])
        rz_float = oracle.forward(n, g, np.array([math.pi / 2]), v)
        np.testing.assert_allclose(rz_float, s_gate, atol=1e-15 * np.abs(v).max() * 4)
        for rot, pauli in (("RX", "X"), ("RY", "Y"), ("RZ", "Z")):
            a = oracle.apply_gate(n, OPS[rot], q, 0, v, -1.0, 0.0)
            b = oracle.apply_gate(n, OPS[pauli], q, 0, v)
            np.testing.assert_array_equal(a, b)


def test_z_expectation_after_single_rotation():
    for th in np.linspace(0, 2 * math.pi, 7):
        for rot in ("RX", "RY"):
            g = W.gates_from_list([(rot, 0, 0)])
            got = oracle.expect(1, g, np.array([th]), [(1.0, "Z")])
            assert abs(got - math.cos(th)) < 1e-15
        g = W.gates_from_list([("RZ", 0, 0)])
        assert oracle.expect(1, g, np.array([th]), [(1.0, "Z")]) == 1.0


def test_dense_route_equals_paper_encode_map_flatten():
    """Sec. III-C route: map_non-CX on each wire's weights, then flatten (Eq. (5)),
    equals flatten first and then the per-gate dense application."""
    n = 3
    rng = np.random.default_rng(8)
    Wt = rng.normal(size=(2, n, 4))
    seq = [(OPS["RX"], 0.3), (OPS["H"], 0.0), (OPS["RZ"], 1.1), (OPS["S"], 0.0), (OPS["RY"], 2.0)]
    Wm = Wt.copy()
    for t in range(Wt.shape[0]):
        for q in range(n):
            w = Wm[t, q]
            for op, th in seq:
                w = oracle.map_noncx(op, w, math.cos(th), math.sin(th))
            Wm[t, q] = w
    via_paper = oracle.expand(Wm)
    v = oracle.expand(Wt)
    for q in range(n):
        for op, th in seq:
            v = oracle.apply_gate(n, op, q, 0, v, math.cos(th), math.sin(th))
    np.testing.assert_allclose(via_paper, v, atol=1e-12)


# ---------------------------------------------------------------- gradients

def test_psr_matches_statevector_finite_differences():
    n = 3
    c = W.random_circuit(n, 40, seed=61)
    obs = W.random_observable(n, 4, seed=62)
    g = oracle.psr_grad(n, c.gates, c.thetas, obs)
    h = 1e-6
    for j in range(c.n_params):
        tp, tm = c.thetas.copy(), c.thetas.copy()
        tp[j] += h
        tm[j] -= h
        fd = (D.statevector_expect(n, c.gates, tp, obs) - D.statevector_expect(n, c.gates, tm, obs)) / (2 * h)
        assert abs(g[j] - fd) < 1e-6 * sum(abs(a) for a, _ in obs)


def test_psr_shared_parameters_sum_over_gates():
    n = 3
    c = W.random_circuit(n, 50, seed=63, shared_params=3)
    obs = W.obs_chain(n)
    g = oracle.psr_grad(n, c.gates, c.thetas, obs)
    per_gate = np.zeros(c.n_params)
    for i in range(c.m):
        if c.gates[i]["op"] >= OPS["RX"]:
            per_gate[c.gates[i]["param"]] += oracle.psr_grad_gate(n, c.gates, c.thetas, obs, i)
    np.testing.assert_allclose(g, per_gate, atol=1e-14)
    h = 1e-6
    for j in range(c.n_params):
        tp, tm = c.thetas.copy(), c.thetas.copy()
        tp[j] += h
        tm[j] -= h
        fd = (D.statevector_expect(n, c.gates, tp, obs) - D.statevector_expect(n, c.gates, tm, obs)) / (2 * h)
        assert abs(g[j] - fd) < 1e-6 * sum(abs(a) for a, _ in obs)


def test_invalid_circuits_rejected():
    g = W.gates_from_list([("CX", 0, 0)])
    with pytest.raises(ValueError):
        oracle.forward(2, g, np.zeros(1), np.zeros(16))
    g = W.gates_from_list([("RX", 0, 5)])
    with pytest.raises(ValueError):
        oracle.forward(2, g, np.zeros(1), np.zeros(16))


# ---------------------------------------------------------------- density matrix

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_density_matrix_against_statevector(n):
    c = W.random_circuit(n, 25 * n, seed=500 + n)
    rho = oracle.density_matrix(n, c.gates, c.thetas)
    U = D.circuit_unitary(n, c.gates, c.thetas)
    psi = U[:, 0]
    np.testing.assert_allclose(rho, np.outer(psi, psi.conj()), atol=1e-12)
    assert abs(np.trace(rho) - 1) < 1e-12
    np.testing.assert_allclose(rho, rho.conj().T, atol=1e-13)
    np.testing.assert_allclose(rho @ rho, rho, atol=1e-12)


def test_density_matrix_equals_product_of_generators_eq2():
    """Eq. (2): rho = 2^-n prod_j (I + S_j) with S_j the evolved generators."""
    n = 3
    c = W.layered_ansatz(n, 60, seed=8)
    gens = oracle.generators(n, c.gates, c.thetas)
    prod = np.eye(2 ** n, dtype=complex)
    for k in range(n):
        Sk = D.coeffs_to_matrix(n, gens[k])
        prod = prod @ (np.eye(2 ** n) + Sk)
    np.testing.assert_allclose(oracle.density_matrix(n, c.gates, c.thetas), prod / 2 ** n,
                               atol=1e-12)
