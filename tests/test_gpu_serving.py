"""Continuous-batching server, both engines (the iteration engine that
advances every admitted request by a slice per persistent launch, and the
per-request context engine): every result is the same served in a mix as
computed alone, and matches the oracle; requests join while others run; a
request that can never fit and a malformed request fail alone; the aging
bound of shortest-work-first admission."""
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


ENGINES = ["iterate", "contexts"]


@pytest.mark.parametrize("engine", ENGINES)
def test_served_results_equal_alone_and_oracle(stab, engine):
    reqs = request_mix(3, 40)
    srv = stab.Server(max_active=8, engine=engine)
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


@pytest.mark.parametrize("engine", ENGINES)
def test_requests_join_while_others_run(stab, engine):
    # a small budget forces queueing: later requests wait for earlier ones to
    # release budget, then are admitted while others are still running
    reqs = request_mix(4, 24)
    fps = [stab.Server.footprint(c, k, o) for c, k, o in reqs]
    srv = stab.Server(max_active=4, hbm_budget=max(fps) * 3, engine=engine)
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


@pytest.mark.parametrize("engine", ENGINES)
def test_oversized_and_malformed_requests_fail_alone(stab, engine):
    good = W.layered_ansatz(4, 100, seed=1)
    big = W.layered_ansatz(10, 50, seed=2)
    bad = W.Circuit(3, W.gates_from_list([("CX", 1, 1)]), np.zeros(0))
    srv = stab.Server(hbm_budget=stab.Server.footprint(big, "expect", W.obs_chain(10)) - 1,
                      engine=engine)
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


@pytest.mark.parametrize("engine", ENGINES)
def test_serving_trace_c5_sampled(stab, engine):
    """The serving workload's own trace (Poisson 2,000/s, n 4..12, depth
    log-uniform 100..60,000, seed 1005): its first 48 requests through the
    server as the bench submits them; those the oracle checks quickly
    (4^n m small) against the oracle -- <O>, and for gradient requests
    sampled slots by the parameter shift."""
    trace = W.serving_trace(48, seed=1005)
    srv = stab.Server(max_active=64, engine=engine)
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


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("policy", ["fifo", "shortest"])
def test_admission_order(stab, policy, engine):
    """One slot: while a blocker runs, a large request and six small ones
    queue.  FIFO admits the large one first; shortest-work-first admits the
    small ones first.  Results are the same under either order."""
    blocker = W.layered_ansatz(9, 1500, seed=1)
    large = W.layered_ansatz(8, 3000, seed=2)
    small = [W.layered_ansatz(3, 40 + k, seed=10 + k) for k in range(6)]
    srv = stab.Server(max_active=1, policy=policy, engine=engine, aging_s=-1.0)
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


@pytest.mark.parametrize("engine", ENGINES)
def test_served_large_gradient_against_oracle(stab, engine):
    """An n = 9 gradient request served in a mix of smaller ones: its <O> and
    sampled slots against the oracle's parameter shift, the others against
    the oracle's <O>."""
    big = W.layered_ansatz(9, 300, seed=909)
    obs = W.obs_chain(9)
    small = request_mix(5, 8)
    srv = stab.Server(max_active=8, engine=engine)
    ids = [srv.submit(c, k, o) for c, k, o in small[:4]]
    ib = srv.submit(big, "grad", obs)
    ids += [srv.submit(c, k, o) for c, k, o in small[4:]]
    rb = srv.wait(ib, timeout_s=300)
    rest = [srv.wait(i, timeout_s=300) for i in ids]
    srv.close()
    assert rb["status"] == 0 and all(r["status"] == 0 for r in rest)
    tol = 1e-12 * l1(obs)
    assert abs(rb["expect"] - oracle.expect(9, big.gates, big.thetas, obs)) <= tol
    rot = [i for i, g in enumerate(big.gates) if int(g["op"]) in W.ROTATIONS]
    rng = np.random.default_rng(19)
    for gi in rng.choice(rot, size=3, replace=False):
        slot = int(big.gates[gi]["param"])
        want = oracle.psr_grad_gate(9, big.gates, big.thetas, obs, int(gi))
        assert abs(rb["grads"][slot] - want) <= tol
    for (c, kind, o), r in zip(small[:4] + small[4:], rest):
        if 4 ** c.n * c.m <= 3e7:
            assert abs(r["expect"] - oracle.expect(c.n, c.gates, c.thetas, o)) <= 1e-12 * l1(o)


def test_iteration_engine_alone_equals_mix_bit_for_bit(stab):
    """The iteration engine runs each request's passes in the same order on
    the same data whatever else shares the launches and however the work is
    sliced: every result (expectation and every gradient entry) served in a
    mix of 32 requests of n = 2..8 (all in the iteration engine) equals, bit for
    bit, the same request served alone with another slice size and another
    shared-memory budget (so some vectors move between shared and global
    memory); all match the oracle and the context engine."""
    rng = np.random.default_rng(77)
    reqs = []
    for k in range(32):
        n = int(rng.integers(2, 9))
        m = int(rng.integers(30, 700 if n <= 6 else 250))
        c = W.layered_ansatz(n, m, seed=7700 + k)
        reqs.append((c, "grad" if k % 2 else "expect", W.obs_chain(n)))
    srv = stab.Server(max_active=64, engine="iterate", iter_chunks=16, iter_max_n=8)
    ids = []
    for k, (c, kind, obs) in enumerate(reqs):
        ids.append(srv.submit(c, kind, obs))
        if k % 8 == 7:
            time.sleep(0.005)
    mix = [srv.wait(i, timeout_s=300) for i in ids]
    srv.close()
    ctx = stab.Server(max_active=64, engine="contexts")
    cids = [ctx.submit(c, kind, obs) for c, kind, obs in reqs]
    via_ctx = [ctx.wait(i, timeout_s=300) for i in cids]
    ctx.close()
    for (c, kind, obs), r, rc in zip(reqs, mix, via_ctx):
        assert r["status"] == 0 and rc["status"] == 0
        one = stab.Server(max_active=1, engine="iterate", iter_chunks=3, iter_max_n=8,
                          iter_smem_kb=64)
        a = one.wait(one.submit(c, kind, obs), timeout_s=300)
        one.close()
        assert a["status"] == 0
        assert a["expect"] == r["expect"]
        tol = 1e-12 * l1(obs)
        assert abs(r["expect"] - oracle.expect(c.n, c.gates, c.thetas, obs)) <= tol
        assert abs(r["expect"] - rc["expect"]) <= tol
        if kind == "grad":
            np.testing.assert_array_equal(a["grads"], r["grads"])
            assert np.abs(r["grads"] - rc["grads"]).max() <= tol
            rot = [i for i, g in enumerate(c.gates) if int(g["op"]) in W.ROTATIONS]
            if rot and 4 ** c.n * c.m <= 2e7:
                gi = int(rot[len(rot) // 2])
                want = oracle.psr_grad_gate(c.n, c.gates, c.thetas, obs, gi)
                assert abs(r["grads"][int(c.gates[gi]["param"])] - want) <= tol


@pytest.mark.parametrize("engine", ENGINES)
def test_shortest_first_with_aging_admits_the_oldest(stab, engine):
    """One slot, shortest-work-first with a 1 ms aging bound: while a blocker
    runs, a large request and six small ones queue; when the slot frees, the
    large request has waited past the bound and is admitted before the small
    ones (without the bound it would come last).  The blocker is long enough
    (15,000 gates at n = 9) that the large request has aged past the bound
    when the slot frees; a blocker done within 1 ms of that submission would
    rightly let a small request in first."""
    blocker = W.layered_ansatz(9, 15000, seed=1)
    large = W.layered_ansatz(8, 3000, seed=2)
    small = [W.layered_ansatz(3, 40 + k, seed=10 + k) for k in range(6)]
    srv = stab.Server(max_active=1, policy="shortest", engine=engine, aging_s=1e-3)
    ib = srv.submit(blocker, "expect", W.obs_chain(9))
    il = srv.submit(large, "expect", W.obs_chain(8))
    isml = [srv.submit(c, "expect", W.obs_chain(3)) for c in small]
    rb = srv.wait(ib, timeout_s=300)
    rl = srv.wait(il, timeout_s=300)
    rs = [srv.wait(i, timeout_s=300) for i in isml]
    srv.close()
    assert rb["status"] == 0 and rl["status"] == 0 and all(r["status"] == 0 for r in rs)
    assert rb["done_s"] - rl["submit_s"] > 1e-3   # the premise: the large one has aged
    assert all(rl["done_s"] <= r["admit_s"] for r in rs)
    assert abs(rl["expect"] - oracle.expect(8, large.gates, large.thetas, W.obs_chain(8))) <= \
        1e-12 * l1(W.obs_chain(8))


@pytest.mark.parametrize("engine", ENGINES)
def test_server_device_memory_goes_through_the_hooks(stab, engine):
    """The server allocates its device memory (request blocks, unit tables,
    contexts' vectors) through the allocator hooks of its options: with
    counting hooks every block is obtained through them and every one is
    handed back by the time the server is destroyed."""
    import ctypes

    import torch
    from paper_2502_10685_gb300 import _lib
    live, calls = {}, {"alloc": 0, "free": 0}

    def _alloc(nbytes, st, user):
        calls["alloc"] += 1
        p = int(torch.cuda.caching_allocator_alloc(int(nbytes), 0))
        live[p] = int(nbytes)
        return p

    def _free(ptr, nbytes, st, user):
        calls["free"] += 1
        assert live.pop(int(ptr)) == int(nbytes)
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _lib.ALLOC_FN(_alloc), _lib.FREE_FN(_free)
    o = _lib.StabServerOpts()
    o.device, o.max_active, o.engine = 0, 8, stab.Server.ENGINES[engine]
    o.alloc, o.free = a, f
    h = ctypes.c_void_p()
    L = _lib.load()
    assert L.stab_server_create(ctypes.byref(o), ctypes.byref(h)) == 0
    reqs = [(W.layered_ansatz(n, 120, seed=90 + n), kind, W.obs_chain(n))
            for n, kind in ((4, "expect"), (5, "grad"), (7, "grad"), (9, "expect"))]
    keep, ids = [], []
    for c, kind, obs in reqs:
        r = stab.Server._request(c, kind, obs, keep)
        i = ctypes.c_int64()
        assert L.stab_serve_submit(h, ctypes.byref(r), ctypes.byref(i)) == 0
        ids.append(i.value)
    done = ctypes.c_int32(0)
    deadline = time.time() + 300
    while not done.value and time.time() < deadline:    # the last request, by polling
        assert L.stab_serve_poll(h, ids[-1], ctypes.byref(done)) == 0
        time.sleep(0.001)
    assert done.value == 1
    for (c, kind, obs), i in zip(reqs, ids):
        res = _lib.StabResult()
        grads = np.zeros(max(c.n_params, 1))
        assert L.stab_server_wait(h, i, 300.0, ctypes.byref(res), grads.ctypes.data) == 0
        assert res.status == 0
        assert abs(res.expect - oracle.expect(c.n, c.gates, c.thetas, obs)) <= 1e-12 * l1(obs)
    assert calls["alloc"] > 0
    assert L.stab_server_destroy(h) == 0
    assert not live and calls["free"] == calls["alloc"]


def test_iteration_engine_deep_gradient_against_oracle(stab):
    """A 60,200-gate n = 4 gradient request through the iteration engine
    (hundreds of slices per unit, both phases of the split sweeps): <O> and
    sampled slots against the oracle's parameter shift, within the 1e-10
    tolerance of circuits of 60K gates and more."""
    c = W.layered_ansatz(4, 60200, seed=1002)
    obs = W.obs_chain(4)
    srv = stab.Server(max_active=4, engine="iterate", iter_chunks=8)
    small = W.layered_ansatz(5, 300, seed=3)
    i_small = srv.submit(small, "grad", W.obs_chain(5))
    i_deep = srv.submit(c, "grad", obs)
    r = srv.wait(i_deep, timeout_s=300)
    r_small = srv.wait(i_small, timeout_s=300)
    srv.close()
    assert r["status"] == 0 and r_small["status"] == 0
    tol = 1e-10 * l1(obs)
    assert abs(r["expect"] - oracle.expect(4, c.gates, c.thetas, obs)) <= tol
    rot = [i for i, g in enumerate(c.gates) if int(g["op"]) in W.ROTATIONS]
    for gi in (rot[0], rot[len(rot) // 2], rot[-1]):
        want = oracle.psr_grad_gate(4, c.gates, c.thetas, obs, gi)
        assert abs(r["grads"][int(c.gates[gi]["param"])] - want) <= tol


def test_iteration_engine_degenerate_requests(stab):
    """Requests the iteration engine must handle without a special path: the
    identity circuit (empty streams), a Clifford-only gradient (no slots),
    one qubit, an observable with an identity term, repeated strings and an
    empty one, random mixed circuits of every opcode with shared slots --
    each against the oracle (gradients by the oracle's parameter shift)."""
    ident = W.Circuit(3, np.zeros(0, dtype=W.GATE_DTYPE), np.zeros(0))
    cliff = W.random_circuit(4, 120, seed=31, clifford_only=True)
    one = W.random_circuit(1, 40, seed=32)
    mixed = W.random_circuit(5, 200, seed=33, shared_params=6)
    obs3 = [(2.5, "III"), (0.5, "ZIZ"), (0.25, "ZIZ"), (-1.0, "XYZ")]
    cases = [(ident, "expect", obs3), (ident, "grad", obs3), (cliff, "grad", W.obs_chain(4)),
             (cliff, "expect", W.obs_chain(4)), (one, "grad", [(1.0, "Z"), (0.5, "X")]),
             (one, "expect", [(1.0, "Y")]), (mixed, "grad", W.random_observable(5, 6, seed=34)),
             (W.layered_ansatz(3, 90, seed=35), "expect", [])]
    srv = stab.Server(max_active=16, engine="iterate", iter_chunks=2)
    ids = [srv.submit(c, kind, obs) for c, kind, obs in cases]
    res = [srv.wait(i, timeout_s=120) for i in ids]
    srv.close()
    for (c, kind, obs), r in zip(cases, res):
        assert r["status"] == 0
        tol = 1e-12 * max(l1(obs), 1.0)
        want = oracle.expect(c.n, c.gates, c.thetas, obs) if obs else 0.0
        assert abs(r["expect"] - want) <= tol, (c.n, kind, r["expect"], want)
        if kind == "grad":
            assert len(r["grads"]) == c.n_params
            if c.n_params:
                ref = oracle.psr_grad(c.n, c.gates, c.thetas, obs)
                assert np.abs(r["grads"] - ref).max() <= tol


@pytest.mark.parametrize("engine", ENGINES)
def test_wait_timeout_then_result_and_destroy_with_requests_in_flight(stab, engine):
    """A wait that gives up (timeout) leaves the request running: a later wait
    returns its result.  Destroying the server with requests still queued or
    running waits for them and releases everything (no hang, no fault)."""
    from paper_2502_10685_gb300._lib import StabError
    big = W.layered_ansatz(8, 6000, seed=71)
    srv = stab.Server(max_active=1, engine=engine)
    i_big = srv.submit(big, "grad", W.obs_chain(8))
    i_next = srv.submit(W.layered_ansatz(4, 300, seed=72), "expect", W.obs_chain(4))
    with pytest.raises(StabError) as err:
        srv.wait(i_next, timeout_s=1e-4)          # still queued behind the large request
    assert err.value.code == -4                     # STAB_E_TIMEOUT
    r = srv.wait(i_next, timeout_s=300)
    assert r["status"] == 0
    c4 = W.layered_ansatz(4, 300, seed=72)
    assert abs(r["expect"] - oracle.expect(4, c4.gates, c4.thetas, W.obs_chain(4))) <= \
        1e-12 * l1(W.obs_chain(4))
    assert srv.wait(i_big, timeout_s=300)["status"] == 0
    # now leave work behind: queued and running requests at destroy time
    for k in range(6):
        srv.submit(W.layered_ansatz(5 + k % 3, 2000, seed=80 + k), "grad", W.obs_chain(5 + k % 3))
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 120
    # the device is still usable afterwards
    s = stab.Stab(3)
    c3 = W.layered_ansatz(3, 50, seed=90)
    s.load_circuit(c3.gates, c3.thetas)
    assert abs(s.expect(W.obs_chain(3)) - oracle.expect(3, c3.gates, c3.thetas, W.obs_chain(3))) \
        <= 1e-12 * l1(W.obs_chain(3))
    s.close()
