"""The sparse term-list path (stab_sparse_*) against the oracles.

Small n: against the dense oracle, including the switch to the dense path.
Large n (up to 32): against the sparse-list oracle, a closed form and
Clifford-only circuits bit for bit.  Also capacity growth, overflow,
determinism, the order history and degenerate inputs.
"""
import math

import numpy as np
import pytest

import layout
import oracle
from paper_2502_10685_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2502_10685_gb300 import stab
    return stab


def l1(obs):
    return sum(abs(c) for c, _ in obs)


def assert_terms_match(n, got_terms, want_keys, want_vals, tol):
    got = layout.terms_to_paper_dict(n, got_terms)
    want = dict(zip([int(k) for k in want_keys], [float(v) for v in want_vals]))
    worst = 0.0
    for k in set(got) | set(want):
        worst = max(worst, abs(got.get(k, 0.0) - want.get(k, 0.0)))
    assert worst <= tol, worst


@pytest.mark.parametrize("n", [2, 4, 6, 8])
def test_generators_vs_dense_oracle(S, n):
    c = W.random_circuit(n, 120, seed=700 + n)
    sp = S.Sparse(n, max_terms=1 << 18)
    sp.load_circuit(c.gates, c.thetas)
    G = oracle.generators(n, c.gates, c.thetas)
    for k in range(n):
        terms, info = sp.generator(k)
        nz = np.nonzero(G[k])[0]
        assert_terms_match(n, terms, nz, G[k][nz], 1e-12)
        assert info["order_final"] == len(terms)
    sp.close()


@pytest.mark.parametrize("n", [3, 5, 8, 10])
def test_expect_vs_dense_oracle_sparse_only_and_switch(S, n):
    c = W.random_circuit(n, 150, seed=720 + n)
    obs = W.random_observable(n, 5, seed=n) + [(0.5, "Z" * n)]
    want = oracle.expect(n, c.gates, c.thetas, obs)
    sp = S.Sparse(n, max_terms=1 << 21)
    sp.load_circuit(c.gates, c.thetas)
    sp.set_dense_threshold(0)
    got, info = sp.expect(obs)
    assert abs(got - want) <= 1e-12 * l1(obs)
    assert info["dense_gates"] == -1
    sp.set_dense_threshold(16)
    got2, info2 = sp.expect(obs)
    assert abs(got2 - want) <= 1e-12 * l1(obs)
    assert info2["dense_gates"] >= 0
    sp.close()


def test_dense_switch_on_layered_ansatz(S):
    n = 8
    c = W.layered_ansatz(n, 400, seed=31)
    obs = W.obs_chain(n)
    want = oracle.expect(n, c.gates, c.thetas, obs)
    sp = S.Sparse(n)
    sp.load_circuit(c.gates, c.thetas)
    got, info = sp.expect(obs)          # default threshold 4^8 / 16
    assert abs(got - want) <= 1e-12 * l1(obs)
    assert 0 < info["dense_gates"] < c.m
    sp.close()


@pytest.mark.parametrize("n", [16, 24, 31, 32])
def test_large_n_vs_sparse_oracle(S, n):
    c = W.clifford_plus_rotations(n, 600, 14, seed=740 + n)
    sp = S.Sparse(n, max_terms=1 << 20)
    sp.load_circuit(c.gates, c.thetas)
    obs = W.obs_chain(n) + W.random_observable(n, 3, seed=n)
    got, info = sp.expect(obs)
    want = oracle.sparse_expect(n, c.gates, c.thetas, obs)
    assert abs(got - want) <= 1e-12 * l1(obs)
    for k in (0, n // 2, n - 1):
        terms, info = sp.generator(k)
        wk, wv = oracle.sparse_generator(n, c.gates, c.thetas, k)
        assert_terms_match(n, terms, wk, wv, 1e-12)
        assert abs(float(np.sum(terms["coeff"] ** 2)) - 1.0) <= 1e-12
    sp.close()


def test_clifford_only_n32_bit_exact(S):
    n = 32
    c = W.clifford_plus_rotations(n, 3000, 0, seed=5)
    sp = S.Sparse(n, max_terms=4096)
    sp.load_circuit(c.gates, c.thetas)
    for k in range(0, n, 5):
        terms, info = sp.generator(k)
        wk, wv = oracle.sparse_generator(n, c.gates, c.thetas, k)
        assert len(terms) == 1 and len(wk) == 1
        assert layout.term_key_paper(n, int(terms[0]["x"]), int(terms[0]["z"])) == int(wk[0])
        assert float(terms[0]["coeff"]) == float(wv[0])
        assert info["order_max"] == 1
    sp.close()


def test_ghz_phase_closed_form_n32(S):
    n = 32
    for phi, q in ((0.37, 0), (2.9, 31)):
        items = [("H", 0)] + [("CX", k, k + 1) for k in range(n - 1)] + [("RZ", q, 0)]
        g = W.gates_from_list(items)
        sp = S.Sparse(n)
        sp.load_circuit(g, np.array([phi]))
        got, _ = sp.expect([(1.0, "X" * n)])
        assert abs(got - math.cos(phi)) <= 1e-14
        got, _ = sp.expect([(1.0, "Z" + "I" * (n - 2) + "Z")])
        assert got == 1.0
        sp.close()


def test_capacity_grows_and_result_is_unchanged(S):
    n = 20
    c = W.clifford_plus_rotations(n, 500, 16, seed=77)
    obs = [(1.0, "Z" * n), (0.5, "X" + "I" * (n - 1))]
    want = oracle.sparse_expect(n, c.gates, c.thetas, obs)
    sp = S.Sparse(n, max_terms=1 << 22)
    sp.load_circuit(c.gates, c.thetas)
    got, info = sp.expect(obs)
    assert abs(got - want) <= 1e-12 * l1(obs)
    if info["order_max"] > 4096:
        assert info["regrows"] >= 1
    terms, ginfo = sp.generator(3)
    wk, wv = oracle.sparse_generator(n, c.gates, c.thetas, 3)
    assert_terms_match(n, terms, wk, wv, 1e-12)
    sp.close()


def test_overflow_is_an_error_not_a_fault(S):
    n = 20
    c = W.clifford_plus_rotations(n, 400, 30, seed=78)   # generator 0 has 64 terms
    sp = S.Sparse(n, max_terms=32)
    sp.load_circuit(c.gates, c.thetas)
    with pytest.raises(S.StabError) as e:
        sp.generator(0)
    assert e.value.code == -2
    with pytest.raises(S.StabError):
        sp.expect([(1.0, "Z" * n)])
    # the context stays usable
    c2 = W.clifford_plus_rotations(n, 100, 2, seed=79)
    sp.load_circuit(c2.gates, c2.thetas)
    got, _ = sp.expect([(1.0, "Z" * n)])
    assert abs(got - oracle.sparse_expect(n, c2.gates, c2.thetas, [(1.0, "Z" * n)])) <= 1e-12
    sp.close()


def test_deterministic_list_order(S):
    n = 24
    c = W.clifford_plus_rotations(n, 500, 14, seed=80)
    sp = S.Sparse(n)
    sp.load_circuit(c.gates, c.thetas)
    a, _ = sp.generator(7)
    b, _ = sp.generator(7)
    assert a.tobytes() == b.tobytes()
    e1, _ = sp.expect(W.obs_chain(n))
    e2, _ = sp.expect(W.obs_chain(n))
    assert e1 == e2
    sp.close()


def test_order_history(S):
    n = 12
    c = W.clifford_plus_rotations(n, 300, 10, seed=81)
    sp = S.Sparse(n)
    sp.load_circuit(c.gates, c.thetas)
    terms, info = sp.generator(0)
    h = sp.order_history()
    assert len(h) == info["steps"]
    assert h[-1] == info["order_final"] == len(terms)
    assert h.max() == info["order_max"]
    rot_steps = sum(int(g["op"]) >= W.OPS["RX"] for g in c.gates)
    assert h.max() <= 2 ** rot_steps
    sp.close()


def test_degenerate_inputs(S):
    n = 9
    sp = S.Sparse(n)
    sp.load_circuit(np.zeros(0, dtype=W.GATE_DTYPE), np.zeros(0))
    assert sp.expect([(2.0, "I" * n)])[0] == 2.0
    assert sp.expect([])[0] == 0.0
    assert sp.expect([(1.0, "X" + "I" * (n - 1))])[0] == 0.0
    terms, info = sp.generator(4)
    assert len(terms) == 1 and int(terms[0]["z"]) == 1 << 4 and float(terms[0]["coeff"]) == 1.0
    c = W.clifford_plus_rotations(n, 50, 3, seed=82)
    sp.load_circuit(c.gates, c.thetas)
    assert sp.expect([(1.0, "I" * n)])[0] == 1.0
    sp.close()


def _runs_and_rotations(n, run, blocks, seed):
    """`blocks` Clifford runs of `run` gates, each followed by one rotation."""
    rng = np.random.default_rng(seed)
    parts, thetas = [], []
    for b in range(blocks):
        c = W.clifford_plus_rotations(n, run, 0, seed=int(rng.integers(1 << 30)))
        parts.append(c.gates)
        r = np.zeros(1, dtype=W.GATE_DTYPE)
        r[0] = (W.OPS[("RX", "RY", "RZ")[b % 3]], int(rng.integers(n)), 0, 0, len(thetas))
        thetas.append(float(rng.uniform(0, 2 * math.pi)))
        parts.append(r)
    return np.concatenate(parts), np.array(thetas)


@pytest.mark.parametrize("n,run", [(8, 23), (8, 24), (8, 300), (32, 71), (32, 72), (32, 500)])
def test_clifford_runs_gate_by_gate_and_tableau(S, n, run):
    """Runs of at least 2n + 8 gates go through the composed tableau, shorter
    runs gate by gate; both against the oracles."""
    gates, th = _runs_and_rotations(n, run, 8, seed=n * 1000 + run)
    sp = S.Sparse(n, max_terms=1 << 16)
    sp.load_circuit(gates, th)
    obs = W.obs_chain(n) + [(0.25, "Y" * n)]
    got, _ = sp.expect(obs)
    if n <= 10:
        want = oracle.expect(n, gates, th, obs)
        G = oracle.generators(n, gates, th)
    else:
        want = oracle.sparse_expect(n, gates, th, obs)
    assert abs(got - want) <= 1e-12 * l1(obs)
    for k in (0, n - 1):
        terms, _ = sp.generator(k)
        if n <= 10:
            nz = np.nonzero(G[k])[0]
            assert_terms_match(n, terms, nz, G[k][nz], 1e-12)
        else:
            wk, wv = oracle.sparse_generator(n, gates, th, k)
            assert_terms_match(n, terms, wk, wv, 1e-12)
    sp.close()


def test_bench_config_n32(S):
    """The bench's term-list workload (n = 32, 20,000 gates, 28 rotations): the
    call succeeds with the order in the millions, repeats bit for bit, and its
    order history is bounded by doubling per rotation; the same circuit family
    with 12 rotations against the sparse oracle."""
    n, m = 32, 20000
    obs = W.obs_chain(n)
    c = W.clifford_plus_rotations(n, m, 28, seed=1006)
    sp = S.Sparse(n, max_terms=1 << 26)
    sp.load_circuit(c.gates, c.thetas)
    v1, info = sp.expect(obs)
    v2, _ = sp.expect(obs)
    assert np.isfinite(v1) and v1 == v2
    assert info["order_max"] > 1_000_000
    h = sp.order_history()
    assert len(h) == info["steps"] and h.max() == info["order_max"]
    assert h.max() <= len(obs) * 2 ** 28
    c12 = W.clifford_plus_rotations(n, m, 12, seed=1006)
    sp.load_circuit(c12.gates, c12.thetas)
    v12, _ = sp.expect(obs)
    assert abs(v12 - oracle.sparse_expect(n, c12.gates, c12.thetas, obs)) <= 1e-12 * l1(obs)
    sp.close()
