"""Continuous-batching server: every result is the same served in a mix as
computed alone, and matches the oracle; requests join while others run; a
request that can never fit and a malformed request fail alone."""
import time

import numpy as np
import pytest

import oracle
from paper_2502_10685_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def l1(obs):
    return sum(abs(a) for a, _ in obs)


@pytest.fixture(scope="module")
def stab():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2502_10685_gb300 import stab as S
    return S


def request_mix(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.integers(2, 10))
        m = int(rng.integers(20, 400 if n <= 6 else 120))
        c = W.layered_ansatz(n, m, seed=seed * 100 + k)
        kind = "expect" if rng.random() < 0.5 else "grad"
        out.append((c, kind, W.obs_chain(n)))
    return out


def alone(stab, c, kind, obs):
    s = stab.Stab(c.n)
    s.load_circuit(c.gates, c.thetas)
    if kind == "expect":
        r = (s.expect(obs), None)
    else:
        r = s.grad(obs)
    s.close()
    return r


def test_served_results_equal_alone_and_oracle(stab):
    reqs = request_mix(3, 40)
    srv = stab.Server(max_active=8)
    ids = []
    for k, (c, kind, obs) in enumerate(reqs):
        ids.append(srv.submit(c, kind, obs))
        if k % 10 == 9:
            time.sleep(0.01)          # later requests arrive while earlier ones run
    res = [srv.wait(i, timeout_s=300) for i in ids]
    srv.close()
    for (c, kind, obs), r in zip(reqs, res):
        assert r["status"] == 0
        e_alone, g_alone = alone(stab, c, kind, obs)
        assert abs(r["expect"] - e_alone) <= 1e-12 * l1(obs)
        if kind == "grad":
            assert np.abs(r["grads"] - g_alone).max() <= 1e-12 * l1(obs)
        if c.n <= 6:
            assert abs(r["expect"] - oracle.expect(c.n, c.gates, c.thetas, obs)) <= 1e-12 * l1(obs)
        assert r["submit_s"] <= r["admit_s"] <= r["done_s"]


def test_requests_join_while_others_run(stab):
    # a small budget forces queueing: later requests wait for earlier ones to
    # release budget, then are admitted while others are still running
    reqs = request_mix(4, 24)
    fps = [stab.Server.footprint(c, k, o) for c, k, o in reqs]
    srv = stab.Server(max_active=4, hbm_budget=max(fps) * 3)
    ids = [srv.submit(c, k, o) for c, k, o in reqs]
    res = [srv.wait(i, timeout_s=300) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["active"] == 0 and st["bytes_in_use"] == 0
    assert all(r["status"] == 0 for r in res)
    admits = sorted(r["admit_s"] for r in res)
    dones = sorted(r["done_s"] for r in res)
    # some request was admitted after another had already completed, and some
    # request was admitted before another admitted earlier had completed
    assert admits[-1] > dones[0]
    overlap = any(a["admit_s"] < b["done_s"] and b["admit_s"] < a["admit_s"]
                  for a in res for b in res)
    assert overlap


def test_oversized_and_malformed_requests_fail_alone(stab):
    good = W.layered_ansatz(4, 100, seed=1)
    big = W.layered_ansatz(10, 50, seed=2)
    bad = W.Circuit(3, W.gates_from_list([("CX", 1, 1)]), np.zeros(0))
    srv = stab.Server(hbm_budget=stab.Server.footprint(big, "expect", W.obs_chain(10)) - 1)
    i_big = srv.submit(big, "expect", W.obs_chain(10))
    i_bad = srv.submit(bad, "expect", W.obs_chain(3))
    i_good = srv.submit(good, "grad", W.obs_chain(4))
    r_big, r_bad, r_good = (srv.wait(i, timeout_s=120) for i in (i_big, i_bad, i_good))
    srv.close()
    assert r_big["status"] == -3      # STAB_E_NOMEM
    assert r_bad["status"] == -1      # STAB_E_INVAL
    assert r_good["status"] == 0
    g_ref = oracle.psr_grad(4, good.gates, good.thetas, W.obs_chain(4))
    assert np.abs(r_good["grads"] - g_ref).max() <= 1e-12 * l1(W.obs_chain(4))


def test_serving_trace_c5_sampled(stab):
    """The serving workload's own trace (Poisson 2,000/s, n 4..12, depth
    log-uniform 100..60,000, seed 1005): its first 48 requests through the
    server as the bench submits them; those the oracle checks quickly
    (4^n m small) against the oracle -- <O>, and for gradient requests
    sampled slots by the parameter shift."""
    trace = W.serving_trace(48, seed=1005)
    srv = stab.Server(max_active=64)
    ids = [srv.submit(r.circuit, r.kind, r.observable) for r in trace]
    res = [srv.wait(i, timeout_s=600) for i in ids]
    srv.close()
    rng = np.random.default_rng(9)
    checked = 0
    for r, out in zip(trace, res):
        assert out["status"] == 0
        assert np.isfinite(out["expect"])
        c, obs = r.circuit, r.observable
        if 4 ** c.n * c.m > 3e7:
            continue
        assert abs(out["expect"] - oracle.expect(c.n, c.gates, c.thetas, obs)) <= 1e-10 * l1(obs)
        if r.kind == "grad" and c.n_params:
            rot = [i for i, g in enumerate(c.gates) if int(g["op"]) in W.ROTATIONS]
            for gi in rng.choice(rot, size=min(3, len(rot)), replace=False):
                slot = int(c.gates[gi]["param"])
                # each slot is read by one gate in this ansatz: PSR of that gate
                want = oracle.psr_grad_gate(c.n, c.gates, c.thetas, obs, int(gi))
                assert abs(out["grads"][slot] - want) <= 1e-10 * l1(obs)
        checked += 1
    assert checked >= 6


@pytest.mark.parametrize("policy", ["fifo", "shortest"])
def test_admission_order(stab, policy):
    """One slot: while a blocker runs, a large request and six small ones
    queue.  FIFO admits the large one first; shortest-work-first admits the
    small ones first.  Results are the same under either order."""
    blocker = W.layered_ansatz(9, 1500, seed=1)
    large = W.layered_ansatz(8, 3000, seed=2)
    small = [W.layered_ansatz(3, 40 + k, seed=10 + k) for k in range(6)]
    srv = stab.Server(max_active=1, policy=policy)
    ib = srv.submit(blocker, "expect", W.obs_chain(9))
    il = srv.submit(large, "expect", W.obs_chain(8))
    isml = [srv.submit(c, "expect", W.obs_chain(3)) for c in small]
    rb = srv.wait(ib, timeout_s=300)
    rl = srv.wait(il, timeout_s=300)
    rs = [srv.wait(i, timeout_s=300) for i in isml]
    srv.close()
    assert rb["status"] == 0 and rl["status"] == 0 and all(r["status"] == 0 for r in rs)
    if policy == "fifo":
        assert all(rl["done_s"] <= r["admit_s"] for r in rs)
    else:
        assert all(r["done_s"] <= rl["admit_s"] for r in rs)
    for c, r in zip(small, rs):
        assert abs(r["expect"] - oracle.expect(3, c.gates, c.thetas, W.obs_chain(3))) <= 1e-12 * l1(W.obs_chain(3))
