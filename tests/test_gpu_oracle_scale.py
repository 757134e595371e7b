"""CUDA path vs the CPU oracle at the sizes the other parity tests do not reach.

* The differentiation workload at full size: n = 8, the 10,000-gate layered
  ansatz (seed 1004), O = sum Z_i Z_{i+1} + 0.5 sum X_i.  The adjoint gradient
  is compared with the oracle's parameter shift (two full propagations per
  slot, exact for these gates, Sec. I) on sampled slots, and <O> with the
  oracle's backward propagation.
* n = 10 gradients and n = 11 generators and <O> on layered circuits of a few
  hundred gates; n = 12 <O> on a 400-gate circuit.
* Deep circuits: the adjoint over the paper-scale 60,200 gates at n = 4 (the
  1e-10 tolerance of circuits of 60K gates and more) and over 20,000 gates at
  n = 6, against the oracle's parameter shift.

Tolerances as in the other parity tests: generators max |a - b| <= 1e-12
(unit 2-norm), <O> and gradients within 1e-12 * sum |o_P|.  The oracle runs
several propagations at once on host threads (ctypes releases the GIL).
"""
import concurrent.futures as cf

import numpy as np
import pytest

import layout
import oracle
from paper_2502_10685_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stab():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2502_10685_gb300 import stab as S
    return S


def l1(obs):
    return sum(abs(a) for a, _ in obs)


def slot_gates(c):
    """{slot: gate index} for circuits whose slots are each read by one gate."""
    out = {}
    for i, g in enumerate(c.gates):
        if int(g["op"]) in W.ROTATIONS:
            assert int(g["param"]) not in out
            out[int(g["param"])] = i
    return out


def oracle_jobs(jobs):
    """Runs the zero-argument callables on host threads, results in order."""
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), 8))) as ex:
        futs = [ex.submit(j) for j in jobs]
        return [f.result() for f in futs]


def check_grad_against_oracle(stab, c, obs, n_slots, seed):
    s = stab.Stab(c.n)
    s.load_circuit(c.gates, c.thetas)
    e, g = s.grad(obs)
    s.close()
    sg = slot_gates(c)
    rng = np.random.default_rng(seed)
    slots = [int(k) for k in rng.choice(sorted(sg), size=min(n_slots, len(sg)), replace=False)]
    jobs = [lambda: oracle.expect(c.n, c.gates, c.thetas, obs)]
    jobs += [(lambda gi=sg[k]: oracle.psr_grad_gate(c.n, c.gates, c.thetas, obs, gi))
             for k in slots]
    ref = oracle_jobs(jobs)
    tol = 1e-12 * l1(obs)
    assert abs(e - ref[0]) <= tol, (e, ref[0])
    for k, want in zip(slots, ref[1:]):
        assert abs(g[k] - want) <= tol, (k, g[k], want)
    return g, slots


def test_c4_full_size_adjoint_against_oracle_psr(stab):
    """n = 8, 10,000 gates, every surviving rotation its own slot: the
    adjoint's entries on 6 sampled slots equal the oracle's parameter shift."""
    c = W.layered_ansatz(8, 10000, seed=1004)
    assert c.m == 10000 and c.n_params > 6000
    g, _ = check_grad_against_oracle(stab, c, W.obs_chain(8), 6, seed=41)
    assert np.all(np.isfinite(g))


def test_n10_gradient_against_oracle_psr(stab):
    c = W.layered_ansatz(10, 400, seed=1010)
    check_grad_against_oracle(stab, c, W.obs_chain(10), 4, seed=42)


def test_n11_generators_and_expectation_against_oracle(stab):
    """n = 11 (4^11 coefficients per vector), 240 gates: three sampled
    generators element by element, every generator's norm, and <O>."""
    n = 11
    c = W.layered_ansatz(n, 240, seed=1111)
    obs = W.obs_chain(n)
    s = stab.Stab(n)
    s.apply_circuit(c.gates, c.thetas)
    gens = s.generators()
    e = s.expect(obs)
    s.close()
    ks = [0, 6, 10]
    jobs = [(lambda k=k: oracle.forward(n, c.gates, c.thetas, oracle.generator(n, k))) for k in ks]
    jobs.append(lambda: oracle.expect(n, c.gates, c.thetas, obs))
    ref = oracle_jobs(jobs)
    for k, want in zip(ks, ref[:-1]):
        got = layout.lib_to_paper(n, gens[k])
        assert np.abs(got - want).max() <= 1e-12, k
    for k in range(n):
        assert abs(float(np.dot(gens[k], gens[k])) - 1.0) <= 1e-12
    assert abs(e - ref[-1]) <= 1e-12 * l1(obs)


def test_n11_streamed_and_plain_expectation_against_oracle(stab):
    n = 11
    c = W.layered_ansatz(n, 200, seed=1112)
    obs = W.random_observable(n, 9, seed=1113)
    ref = oracle.expect(n, c.gates, c.thetas, obs)
    for kernel in ("streamed", "plain"):
        s = stab.Stab(n, kernel=kernel)
        s.load_circuit(c.gates, c.thetas)
        got = s.expect(obs)
        s.close()
        assert abs(got - ref) <= 1e-12 * l1(obs), kernel


def test_n12_expectation_400_gates_against_oracle(stab):
    """n = 12, the largest register, 400 gates (24 layers and a partial one)."""
    n = 12
    c = W.layered_ansatz(n, 400, seed=1212)
    obs = W.obs_chain(n)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    got = s.expect(obs)
    s.close()
    ref = oracle.expect(n, c.gates, c.thetas, obs)
    assert abs(got - ref) <= 1e-12 * l1(obs)


def test_deep_gradient_n4_60200_against_oracle_psr(stab):
    """The paper-scale depth: n = 4, the 60,200-gate layered ansatz.  The
    adjoint carries lambda and rho backward through the inverse maps over
    all 60,200 gates; its entries on 8 sampled slots against the oracle's
    parameter shift (the 1e-10 tolerance of circuits of 60K gates and more),
    and <O> against the oracle."""
    c = W.layered_ansatz(4, 60200, seed=1002)
    obs = W.obs_chain(4)
    s = stab.Stab(4)
    s.load_circuit(c.gates, c.thetas)
    e, g = s.grad(obs)
    s.close()
    sg = slot_gates(c)
    rng = np.random.default_rng(43)
    keys = sorted(sg)
    # both ends of the circuit and around the middle, where the split sweeps meet
    picks = [keys[0], keys[1], keys[len(keys) // 2 - 1], keys[len(keys) // 2],
             keys[len(keys) // 2 + 1], keys[-2], keys[-1]]
    picks += [int(k) for k in rng.choice(keys, size=1)]
    jobs = [lambda: oracle.expect(4, c.gates, c.thetas, obs)]
    jobs += [(lambda gi=sg[k]: oracle.psr_grad_gate(4, c.gates, c.thetas, obs, gi))
             for k in picks]
    ref = oracle_jobs(jobs)
    tol = 1e-10 * l1(obs)
    assert abs(e - ref[0]) <= tol
    for k, want in zip(picks, ref[1:]):
        assert abs(g[k] - want) <= tol, (k, g[k], want)


def test_deep_gradient_n6_20000_against_oracle_psr(stab):
    """n = 6, 20,000 gates (the deepest circuits of the batch workload): the
    adjoint against the oracle's parameter shift on 4 sampled slots."""
    c = W.layered_ansatz(6, 20000, seed=1006)
    check_grad_against_oracle(stab, c, W.obs_chain(6), 4, seed=44)
