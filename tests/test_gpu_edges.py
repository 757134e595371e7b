"""Edge cases through the C interface: identity circuits, n = 1, empty and
degenerate observables, circuits without angles, parameter updates from the
device, and batches holding all of these."""
import math

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
        pytest.fail("CUDA device required")
    from paper_2502_10685_gb300 import stab as S
    return S


def empty_circuit(n):
    return W.Circuit(n, np.zeros(0, dtype=W.GATE_DTYPE), np.zeros(0))


@pytest.mark.parametrize("n", [1, 3, 7])
def test_observable_identity_duplicates_and_empty(stab, n):
    c = W.layered_ansatz(n, 60, seed=n) if n > 1 else W.random_circuit(1, 20, seed=1)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    ident = "I" * n
    assert abs(s.expect([(2.5, ident)]) - 2.5) <= 1e-14          # <I> = 1 for any U
    zz = "Z" + "I" * (n - 1)
    dup = s.expect([(0.5, zz), (0.25, zz), (0.25, zz)])          # equal strings are merged
    assert abs(dup - s.expect([(1.0, zz)])) <= 1e-14
    assert abs(dup - oracle.expect(n, c.gates, c.thetas, [(1.0, zz)])) <= 1e-12
    assert s.expect([]) == 0.0                                    # empty observable
    s.close()


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_identity_circuit_all_entry_points(stab, n):
    c = empty_circuit(n)
    s = stab.Stab(n)
    s.apply_circuit(c.gates, c.thetas)
    g = layout.lib_to_paper(n, s.generators())
    np.testing.assert_array_equal(g, oracle.generators(n, c.gates, c.thetas))
    obs = [(1.0, "Z" * n)]
    assert s.expect(obs) == 1.0
    e, grads = s.grad(obs)
    assert e == 1.0 and grads.size == 0
    rho = s.density_matrix()
    assert rho[0, 0] == 1.0 and np.count_nonzero(rho) == 1
    s.close()


def test_clifford_only_gradient_has_no_slots(stab):
    c = W.random_circuit(4, 100, seed=3, clifford_only=True)
    s = stab.Stab(4)
    s.load_circuit(c.gates, c.thetas)
    e, g = s.grad(W.obs_chain(4))
    s.close()
    assert g.size == 0
    assert abs(e - oracle.expect(4, c.gates, c.thetas, W.obs_chain(4))) <= 1e-12 * 7.5


@pytest.mark.parametrize("n", [4, 6, 8])
def test_device_parameter_updates_then_generators(stab, n):
    import torch
    c = W.layered_ansatz(n, 80 * (9 - n), seed=40 + n)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    for shift in (0.0, 0.7, -1.9):
        th = c.thetas + shift
        s.set_params(torch.tensor(th, device="cuda"))
        s.run_generators()
        got = layout.lib_to_paper(n, s.generators())
        assert np.abs(got - oracle.generators(n, c.gates, th)).max() <= 1e-12
    s.close()


def test_angles_far_outside_one_turn(stab):
    """Angle reduction: theta and theta + 2 pi k give the same map (to the
    rounding of the reduction), at both signs and large |k|."""
    c = W.layered_ansatz(3, 90, seed=5)
    s = stab.Stab(3)
    s.load_circuit(c.gates, c.thetas)
    ref = s.expect(W.obs_chain(3))
    for k in (-40, -1, 1, 40):
        s.set_params(c.thetas + 2 * math.pi * k)
        assert abs(s.expect(W.obs_chain(3)) - ref) <= 1e-11
    s.close()


def test_batch_with_degenerate_items(stab):
    items = [
        W.BatchItem(empty_circuit(1), "generators"),
        W.BatchItem(empty_circuit(6), "expect", [(1.0, "Z" * 6)]),
        W.BatchItem(W.random_circuit(1, 40, seed=2), "expect", [(1.0, "Z")]),
        W.BatchItem(W.layered_ansatz(8, 30, seed=3), "generators"),
        W.BatchItem(W.layered_ansatz(5, 200, seed=4), "expect", []),
    ]
    b = stab.Batch(items)
    b.run()
    ex = b.expectations()
    assert ex[1] == 1.0 and ex[4] == 0.0
    c = items[2].circuit
    assert abs(ex[2] - oracle.expect(1, c.gates, c.thetas, [(1.0, "Z")])) <= 1e-12
    for k in (0, 3):
        c = items[k].circuit
        got = layout.lib_to_paper(c.n, b.generators(k))
        assert np.abs(got - oracle.generators(c.n, c.gates, c.thetas)).max() <= 1e-12
    b.close()


def test_server_small_and_large_requests_mixed(stab):
    srv = stab.Server(max_active=16)
    reqs = []
    for k in range(12):
        n = 1 if k % 3 == 0 else (10 if k % 3 == 1 else 5)
        c = W.random_circuit(1, 30, seed=k) if n == 1 else W.layered_ansatz(n, 30 + k, seed=k)
        kind = "grad" if k % 2 else "expect"
        reqs.append((c, kind, W.obs_chain(n) if n > 1 else [(1.0, "Z")]))
    ids = [srv.submit(*r) for r in reqs]
    res = [srv.wait(i, timeout_s=300) for i in ids]
    srv.close()
    for (c, kind, obs), r in zip(reqs, res):
        assert r["status"] == 0
        ref = oracle.expect(c.n, c.gates, c.thetas, obs) if c.n <= 6 else None
        if ref is not None:
            assert abs(r["expect"] - ref) <= 1e-12 * sum(abs(a) for a, _ in obs)


def test_contexts_of_different_sizes_interleaved(stab):
    # The persistent batch kernel serves contexts of every n <= 6 with a
    # shared-memory size of its own; a small context set up after a large one
    # must not shrink the large one's launch limit.
    ctxs = []
    for n in (6, 2, 5, 3):
        c = W.layered_ansatz(n, 400, seed=40 + n)
        s = stab.Stab(n)
        s.load_circuit(c.gates, c.thetas)
        ctxs.append((s, c))
    for _ in range(2):
        for s, c in ctxs:
            obs = W.obs_chain(c.n)
            ref = oracle.expect(c.n, c.gates, c.thetas, obs)
            assert abs(s.expect(obs) - ref) <= 1e-12 * sum(abs(a) for a, _ in obs)
            s.apply_circuit(c.gates, c.thetas)
            g = layout.lib_to_paper(c.n, s.generators())
            assert np.abs(g - oracle.generators(c.n, c.gates, c.thetas)).max() <= 1e-12
    for s, _ in ctxs:
        s.close()


@pytest.mark.parametrize("n", [3, 4, 6, 8])
def test_interleaved_async_calls(stab, n):
    # Generators on the context stream while observables are swapped and
    # expectations and gradients queued on the other stream: each result
    # must be that of its own observable and of the circuit loaded last.
    import torch
    c1 = W.layered_ansatz(n, 600 if n <= 6 else 200, seed=900 + n)
    c2 = W.layered_ansatz(n, 600 if n <= 6 else 200, seed=950 + n)
    obs = [W.obs_chain(n), W.obs_z(n, 0), W.random_observable(n, 4, seed=9 + n)]
    s = stab.Stab(n)
    out = torch.zeros(len(obs), dtype=torch.float64, device="cuda")
    got = {}
    for c in (c1, c2):
        s.load_circuit(c.gates, c.thetas)
        s.run_generators()
        for k, o in enumerate(obs):
            s.set_observable(o)
            s.expect_async(out[k:k + 1])
        g = torch.zeros(max(c.n_params, 1), dtype=torch.float64, device="cuda")
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.grad_async(e, g)
        s.synchronize()
        got[id(c)] = (out.cpu().numpy().copy(), s.generators(), float(e[0]))
    s.close()
    for c in (c1, c2):
        ex, gens, e_grad = got[id(c)]
        for k, o in enumerate(obs):
            ref = oracle.expect(n, c.gates, c.thetas, o)
            assert abs(ex[k] - ref) <= 1e-12 * sum(abs(a) for a, _ in o)
        ref_last = oracle.expect(n, c.gates, c.thetas, obs[-1])
        assert abs(e_grad - ref_last) <= 1e-12 * sum(abs(a) for a, _ in obs[-1])
        if n <= 6:
            ref_g = oracle.generators(n, c.gates, c.thetas)
            assert np.abs(layout.lib_to_paper(n, gens) - ref_g).max() <= 1e-12


@pytest.mark.parametrize("n,m", [(2, 8 * 32), (2, 8 * 40), (3, 12 * 25)])
def test_chain_edges(stab, n, m):
    # the shortest plans that still cut into K >= 3 parts, an observable with
    # an identity term and a repeated string, and a Clifford-only stretch
    base = W.layered_ansatz(n, m, seed=700 + m)
    cliff = W.random_circuit(n, 200, seed=701 + m, clifford_only=True)
    g = np.concatenate([base.gates, cliff.gates, base.gates])
    th = np.concatenate([base.thetas, base.thetas + 0.25])
    g = g.copy()
    off = len(base.gates) + len(cliff.gates)
    rot = np.isin(g["op"][off:], [W.OPS[r] for r in ("RX", "RY", "RZ")])
    g["param"][off:][rot] += base.n_params
    c = W.Circuit(n, g, th)
    obs = [(0.5, "I" * n), (1.0, "Z" + "I" * (n - 1)), (0.25, "Z" + "I" * (n - 1)),
           (-0.75, "X" * n)]
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    cut, vectors, eu = s.split_info()
    ref = oracle.expect(n, c.gates, c.thetas, obs)
    assert abs(s.expect(obs) - ref) <= 1e-12 * sum(abs(a) for a, _ in obs)
    s.run_generators()
    got = layout.lib_to_paper(n, s.generators())
    assert np.abs(got - oracle.generators(n, c.gates, c.thetas)).max() <= 1e-12
    s.close()


def test_fp64_probe_measures_a_plausible_rate(stab):
    """The roofline's denominator: DFMA and FP64 MMA chains give a positive
    rate below the GPU's nominal FP64 peak (152 SMs x 4 flop/clk x 2.07 GHz
    = 1.26 TFLOP/s on a GB300, with a margin for other parts), and a longer
    launch takes proportionally longer."""
    tf1, ms1 = stab.stab_probe_fp64("dfma", 1024)
    tf2, ms2 = stab.stab_probe_fp64("dfma", 4096)
    tm, _ = stab.stab_probe_fp64("dmma", 512)
    for tf in (tf1, tf2, tm):
        assert 0.05 < tf < 3.0
    assert 2.5 < ms2 / ms1 < 6.0


def test_pass_probe_measures_plausible_latencies(stab):
    """The register pass loop's pieces: every pattern gives a positive cycle
    count per pass, a wire pass costs at least the three dependent FP64
    instructions' latency, and adding shared-memory round trips to the same
    passes does not make them cheaper."""
    c0 = stab.stab_probe_pass(0, 256, 4000)
    c1 = stab.stab_probe_pass(1, 256, 4000)
    c2 = stab.stab_probe_pass(2, 256, 4000)
    c3 = stab.stab_probe_pass(3, 128, 4000)
    for c in (c0, c1, c2, c3, stab.stab_probe_pass(0, 128, 4000), stab.stab_probe_pass(4, 256, 4000)):
        assert 30.0 < c < 1e5
    assert c1 >= 0.95 * c0 and c2 >= 0.95 * c1


def test_no_device_memory_growth_over_repeated_use(stab):
    """Contexts, batches and servers created, used and destroyed over and over:
    every block taken through the PyTorch allocator hooks is handed back
    (torch's allocated bytes return to where they started) and the device's
    free memory does not drift."""
    import torch
    from paper_2502_10685_gb300 import workloads as W2

    def cycle(k):
        c = W2.layered_ansatz(5, 300, seed=500 + k)
        s = stab.Stab(5)
        s.apply_circuit(c.gates, c.thetas)
        s.generators()
        s.grad(W2.obs_chain(5))
        s.close()
        items = [W2.BatchItem(W2.layered_ansatz(n, 200, seed=510 + k + n), "expect",
                              W2.obs_chain(n)) for n in (3, 6, 8)]
        b = stab.Batch(items)
        b.run()
        b.expectations()
        b.close()
        srv = stab.Server(max_active=4)
        ids = [srv.submit(W2.layered_ansatz(n, 150, seed=520 + k + n), kind, W2.obs_chain(n))
               for n, kind in ((4, "grad"), (6, "expect"), (9, "grad"))]
        for i in ids:
            assert srv.wait(i, timeout_s=120)["status"] == 0
        srv.close()

    cycle(0)                                   # first use: tuning, pools, caches
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(1, 9):
        cycle(k)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < (256 << 20), (free0 - free1)
