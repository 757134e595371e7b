"""CUDA path vs the CPU oracle, element by element, through the C interface.

Tolerances (the stated 1e-12 relative, 1e-10 after 60K gates, applied per vector): generators
max |a - b| <= tol * ||b||_2 (= tol, generators have unit norm); <O> within
tol * sum |o_P|; tol = 1e-12, or 1e-10 for circuits of 60K gates and more.
Clifford-only circuits must match bit for bit.
"""
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
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2502_10685_gb300 import stab as S
    return S


def tol_for(m):
    return 1e-10 if m >= 60000 else 1e-12


def run_gens(S, c, kernel="auto", fuse=True):
    s = S.Stab(c.n, kernel=kernel, fuse=fuse)
    s.apply_circuit(c.gates, c.thetas)
    g = s.generators()
    s.close()
    return layout.lib_to_paper(c.n, g)


def obs_l1(obs):
    return sum(abs(a) for a, _ in obs)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("kernel", ["auto", "streamed", "plain"])
def test_generators_random_circuits(stab, n, kernel):
    m = 150 if n <= 6 else 60
    c = W.random_circuit(n, m, seed=1000 + n)
    ref = oracle.generators(n, c.gates, c.thetas)
    got = run_gens(stab, c, kernel)
    assert np.abs(got - ref).max() <= 1e-12


@pytest.mark.parametrize("n", [2, 4, 6, 7, 8, 9])
def test_clifford_circuits_bit_exact(stab, n):
    c = W.random_circuit(n, 200, seed=2000 + n, clifford_only=True)
    ref = oracle.generators(n, c.gates, c.thetas)
    for kernel in ("auto", "streamed"):
        got = run_gens(stab, c, kernel)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_expectation_random(stab, n):
    m = 200 if n <= 6 else 60
    c = W.random_circuit(n, m, seed=3000 + n)
    obs = W.random_observable(n, 6, seed=n)
    ref = oracle.expect(n, c.gates, c.thetas, obs)
    for kernel in ("auto", "streamed", "plain"):
        s = stab.Stab(n, kernel=kernel)
        s.load_circuit(c.gates, c.thetas)
        got = s.expect(obs)
        s.close()
        assert abs(got - ref) <= 1e-12 * obs_l1(obs), kernel


def test_config_small_layered_n4_2000(stab):
    """n=4, 2,000-gate layered ansatz: all 4 x 256 coefficients and <Z_0>."""
    c = W.layered_ansatz(4, 2000, seed=1001)
    ref = oracle.generators(4, c.gates, c.thetas)
    s = stab.Stab(4)
    s.apply_circuit(c.gates, c.thetas)
    got = layout.lib_to_paper(4, s.generators())
    assert np.abs(got - ref).max() <= 1e-12
    obs = W.obs_z(4, 0)
    assert abs(s.expect(obs) - oracle.expect(4, c.gates, c.thetas, obs)) <= 1e-12
    s.close()


def test_config_paper_scale_n4_60200(stab):
    """n=4, 60,200 gates: generators and <Z_0 Z_1> within 1e-10."""
    c = W.layered_ansatz(4, 60200, seed=1002)
    ref = oracle.generators(4, c.gates, c.thetas)
    s = stab.Stab(4)
    s.apply_circuit(c.gates, c.thetas)
    got = layout.lib_to_paper(4, s.generators())
    assert np.abs(got - ref).max() <= 1e-10
    obs = W.obs_zz(4, 0, 1)
    assert abs(s.expect(obs) - oracle.expect(4, c.gates, c.thetas, obs)) <= 1e-10
    s.close()


@pytest.mark.parametrize("n,layers,repeats", [(3, 40, 40), (4, 30, 100), (7, 6, 40)])
def test_paper_shaped_long_runs(stab, n, layers, repeats):
    """Runs of 120-300 rotations per wire: each run's map is composed by a
    warp (chunks per lane, ordered product tree) -- through the split sweeps
    at n = 3, 4 and the streamed encode at n = 7."""
    c = W.paper_shaped_ansatz(n, layers, repeats, seed=70 + n)
    ref = oracle.generators(n, c.gates, c.thetas)
    obs = W.obs_chain(n)
    s = stab.Stab(n)
    s.apply_circuit(c.gates, c.thetas)
    got = layout.lib_to_paper(n, s.generators())
    assert np.abs(got - ref).max() <= 1e-12
    assert abs(s.expect(obs) - oracle.expect(n, c.gates, c.thetas, obs)) <= 1e-12 * obs_l1(obs)
    s.close()


def test_paper_shaped_ansatz_fused_maps(stab):
    """W_chain + ZXZ with many repeats: wire runs compose into 3x3 maps."""
    c = W.paper_shaped_ansatz(4, 5, 20, seed=7)
    ref = oracle.generators(4, c.gates, c.thetas)
    for kernel in ("auto", "streamed", "plain"):
        got = run_gens(stab, c, kernel)
        assert np.abs(got - ref).max() <= 1e-12, kernel


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_gradient_matches_psr(stab, n):
    c = W.random_circuit(n, 60, seed=4000 + n)
    obs = W.random_observable(n, 5, seed=40 + n)
    gref = oracle.psr_grad(n, c.gates, c.thetas, obs)
    eref = oracle.expect(n, c.gates, c.thetas, obs)
    for kernel in ("auto", "streamed"):
        s = stab.Stab(n, kernel=kernel)
        s.load_circuit(c.gates, c.thetas)
        e, g = s.grad(obs)
        s.close()
        assert abs(e - eref) <= 1e-12 * obs_l1(obs)
        assert np.abs(g - gref).max() <= 1e-12 * obs_l1(obs), kernel


def test_gradient_shared_parameters(stab):
    c = W.random_circuit(4, 80, seed=51, shared_params=5)
    obs = W.obs_chain(4)
    gref = oracle.psr_grad(4, c.gates, c.thetas, obs)
    s = stab.Stab(4)
    s.load_circuit(c.gates, c.thetas)
    _, g = s.grad(obs)
    s.close()
    assert np.abs(g - gref).max() <= 1e-12 * obs_l1(obs)


@pytest.mark.parametrize("n", [2, 4, 5, 6])
def test_gradient_split_resident(stab, n):
    # long enough for the meet-in-the-middle adjoint (rho_0 and O meet at the
    # cut, then the pair sweeps both parts); shared slots put gates of one
    # parameter on both sides of the cut
    c = W.random_circuit(n, 400, seed=4100 + n, shared_params=7)
    obs = W.random_observable(n, 5, seed=41 + n)
    gref = oracle.psr_grad(n, c.gates, c.thetas, obs)
    eref = oracle.expect(n, c.gates, c.thetas, obs)
    out = {}
    for kernel in ("auto", "resident"):
        s = stab.Stab(n, kernel=kernel)
        s.load_circuit(c.gates, c.thetas)
        out[kernel] = s.grad(obs)
        s.close()
    for kernel, (e, g) in out.items():
        assert abs(e - eref) <= 1e-12 * obs_l1(obs), kernel
        assert np.abs(g - gref).max() <= 1e-12 * obs_l1(obs), kernel


def test_gradient_n8_sampled_psr_and_fd(stab):
    """n=8 layered ansatz, chain observable: adjoint vs oracle PSR on sampled
    gates, and vs central finite differences (h = 1e-6) of the GPU <O>."""
    c = W.layered_ansatz(8, 600, seed=1004)
    obs = W.obs_chain(8)
    s = stab.Stab(8)
    s.load_circuit(c.gates, c.thetas)
    e, g = s.grad(obs)
    assert abs(e - oracle.expect(8, c.gates, c.thetas, obs)) <= 1e-12 * obs_l1(obs)
    rot = [i for i in range(c.m) if c.gates[i]["op"] >= 8]
    rng = np.random.default_rng(0)
    for i in rng.choice(rot, size=3, replace=False):
        j = int(c.gates[i]["param"])
        gp = oracle.psr_grad_gate(8, c.gates, c.thetas, obs, int(i))
        assert abs(g[j] - gp) <= 1e-12 * obs_l1(obs)
    h = 1e-6
    for j in rng.choice(c.n_params, size=3, replace=False):
        tp, tm = c.thetas.copy(), c.thetas.copy()
        tp[j] += h
        tm[j] -= h
        s.set_params(tp)
        fp = s.expect(obs)
        s.set_params(tm)
        fm = s.expect(obs)
        assert abs(g[j] - (fp - fm) / (2 * h)) <= 1e-6 * obs_l1(obs)
    s.close()


def test_identity_circuit_and_n1(stab):
    c = W.Circuit(3, np.zeros(0, dtype=W.GATE_DTYPE), np.zeros(0))
    got = run_gens(stab, c)
    ref = oracle.generators(3, c.gates, c.thetas)
    np.testing.assert_array_equal(got, ref)
    c1 = W.random_circuit(1, 50, seed=3)
    np.testing.assert_allclose(run_gens(stab, c1), oracle.generators(1, c1.gates, c1.thetas),
                               atol=1e-14)


def test_n12_one_generator_sampled(stab):
    """Largest register: n = 12 (4^12 coefficients per vector), short circuit."""
    n = 12
    c = W.layered_ansatz(n, 40, seed=12)
    s = stab.Stab(n)
    s.apply_circuit(c.gates, c.thetas)
    g = s.generators()
    s.close()
    ref = oracle.forward(n, c.gates, c.thetas, oracle.generator(n, 5))
    got = layout.lib_to_paper(n, g[5])
    assert np.abs(got - ref).max() <= 1e-12
    for k in range(n):
        assert abs(np.dot(g[k], g[k]) - 1.0) < 1e-12


def test_set_params_device_tensor(stab):
    import torch
    c = W.layered_ansatz(5, 300, seed=77)
    obs = W.obs_chain(5)
    s = stab.Stab(5)
    s.load_circuit(c.gates, c.thetas)
    th2 = c.thetas + 0.3
    s.set_params(torch.tensor(th2, device="cuda"))
    got = s.expect(obs)
    s.close()
    assert abs(got - oracle.expect(5, c.gates, th2, obs)) <= 1e-12 * obs_l1(obs)


def test_invalid_inputs_return_errors(stab):
    from paper_2502_10685_gb300._lib import StabError
    s = stab.Stab(3)
    bad = W.gates_from_list([("CX", 1, 1)])
    with pytest.raises(StabError) as ei:
        s.load_circuit(bad, np.zeros(0))
    assert ei.value.code == -1
    bad = W.gates_from_list([("RX", 0, 4)])
    with pytest.raises(StabError) as ei:
        s.load_circuit(bad, np.zeros(2))
    assert ei.value.code == -2
    bad = W.gates_from_list([("RX", 0, 0)])
    with pytest.raises(StabError) as ei:
        s.load_circuit(bad, np.array([np.nan]))
    assert ei.value.code == -5
    with pytest.raises(StabError) as ei:
        s.expect([(1.0, "ZII")])
    assert ei.value.code == -7
    s.close()
    with pytest.raises(StabError):
        stab.Stab(13)


def test_deterministic_repeat(stab):
    c = W.layered_ansatz(6, 1000, seed=5)
    a = run_gens(stab, c)
    b = run_gens(stab, c)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7])
def test_long_two_qubit_clifford_runs(stab, n):
    """Runs of 150 consecutive CX/CZ gates between rotation layers (the
    resident kernels split them across several pull passes)."""
    rng = np.random.default_rng(n)
    items, slot = [], 0
    for _ in range(3):
        for _ in range(150):
            a = int(rng.integers(n))
            b = int((a + 1 + rng.integers(n - 1)) % n)
            items.append(("CX" if rng.random() < 0.7 else "CZ", a, b))
        for q in range(n):
            items.append(("RY", q, slot))
            slot += 1
    c = W.Circuit(n, W.gates_from_list(items), rng.uniform(0, 2 * math.pi, slot))
    ref = oracle.generators(n, c.gates, c.thetas)
    for kernel in ("auto", "streamed"):
        got = run_gens(stab, c, kernel)
        assert np.abs(got - ref).max() <= 1e-12, kernel
    obs = W.obs_chain(n)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    e, g = s.grad(obs)
    s.close()
    assert abs(e - oracle.expect(n, c.gates, c.thetas, obs)) <= 1e-12 * obs_l1(obs)
    gref = oracle.psr_grad(n, c.gates, c.thetas, obs)
    assert np.abs(g - gref).max() <= 1e-12 * obs_l1(obs)


def test_autograd_function_matches_psr(stab):
    import torch
    from paper_2502_10685_gb300.autograd import ExpectationLayer
    c = W.layered_ansatz(4, 300, seed=8)
    obs = W.obs_chain(4)
    layer = ExpectationLayer(c, obs)
    f = layer()
    f.backward()
    g = layer.thetas.grad.detach().cpu().numpy()
    gref = oracle.psr_grad(4, c.gates, c.thetas, obs)
    assert abs(float(f) - oracle.expect(4, c.gates, c.thetas, obs)) <= 1e-12 * obs_l1(obs)
    assert np.abs(g - gref).max() <= 1e-12 * obs_l1(obs)
    # one optimizer step moves <O> the way the gradient says
    opt = torch.optim.SGD([layer.thetas], lr=1e-3)
    opt.step()
    f2 = float(layer())
    assert f2 < float(f) + 1e-15


def test_bounded_wait_reports_timeout_and_device_stays_usable(stab):
    """A device wait that nothing completes gives up after its poll bound and
    the host reads STAB_E_TIMEOUT; later work on the device is unaffected."""
    from paper_2502_10685_gb300 import _lib
    L = _lib.load()
    assert L.stab_selftest_bounded_wait(0) == 0
    assert L.stab_selftest_bounded_wait(20000) == -4      # STAB_E_TIMEOUT
    c = W.layered_ansatz(3, 100, seed=9)
    got = run_gens(stab, c)
    assert np.abs(got - oracle.generators(3, c.gates, c.thetas)).max() <= 1e-12


def _bitrev_perm(n):
    idx = np.arange(2 ** n)
    out = np.zeros_like(idx)
    for q in range(n):
        out |= ((idx >> q) & 1) << (n - 1 - q)
    return out


@pytest.mark.parametrize("n", [1, 2, 4, 5, 6, 7, 8])
def test_density_matrix_against_oracle(stab, n):
    """Decoded rho (library: bit q = qubit q) vs the oracle's Sec. III-D decode
    (qubit 0 most significant)."""
    c = W.layered_ansatz(n, 40 * n, seed=600 + n) if n > 1 else W.random_circuit(1, 30, seed=6)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    rho = s.density_matrix()
    s.close()
    perm = _bitrev_perm(n)
    got = rho[np.ix_(perm, perm)]
    ref = oracle.density_matrix(n, c.gates, c.thetas)
    assert np.abs(got - ref).max() <= 1e-12
    assert abs(np.trace(rho) - 1) <= 1e-12


@pytest.mark.parametrize("n", [2, 3, 4])
def test_density_matrix_split_sweep(stab, n):
    """Long circuits: rho_0 through the first part, then the second part's
    transfer matrix (the split sweep of the generators), decoded."""
    c = W.layered_ansatz(n, 2000, seed=610 + n)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    assert s.split_info()[0] > 0
    rho = s.density_matrix()
    s.close()
    perm = _bitrev_perm(n)
    ref = oracle.density_matrix(n, c.gates, c.thetas)
    assert np.abs(rho[np.ix_(perm, perm)] - ref).max() <= 1e-12
    assert abs(np.trace(rho) - 1) <= 1e-12


@pytest.mark.parametrize("n,m", [(2, 4000), (3, 6000)])
def test_chain_of_transfer_matrices(stab, n, m):
    """n <= 3, long circuits: cut into K >= 3 parts; the generators, rho and
    <O> go through the chain of the later parts' transfer matrices.  <O> alone
    runs the sweep itself; after the generators it reuses theirs; new angles
    must not reuse a sweep made for the old ones."""
    c = W.layered_ansatz(n, m, seed=620 + n)
    obs = W.random_observable(n, 5, seed=62 + n)
    l1 = sum(abs(a) for a, _ in obs)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    cut, vectors, expect_units = s.split_info()
    assert cut > 0 and expect_units == 0
    assert vectors >= n + 1 + 2 * (4 ** n - 1)          # at least two transfer matrices
    assert abs(s.expect(obs) - oracle.expect(n, c.gates, c.thetas, obs)) <= 1e-12 * l1
    s.run_generators()
    assert abs(s.expect(W.obs_chain(n)) - oracle.expect(n, c.gates, c.thetas, W.obs_chain(n))) \
        <= 1e-12 * sum(abs(a) for a, _ in W.obs_chain(n))
    got = layout.lib_to_paper(n, s.generators())
    assert np.abs(got - oracle.generators(n, c.gates, c.thetas)).max() <= 1e-12
    rho = s.density_matrix()
    perm = _bitrev_perm(n)
    assert np.abs(rho[np.ix_(perm, perm)] - oracle.density_matrix(n, c.gates, c.thetas)).max() \
        <= 1e-12
    th2 = np.random.default_rng(5).uniform(0, 2 * np.pi, c.n_params)
    s.set_params(th2)
    assert abs(s.expect(obs) - oracle.expect(n, c.gates, th2, obs)) <= 1e-12 * l1
    s.run_generators()
    got = layout.lib_to_paper(n, s.generators())
    assert np.abs(got - oracle.generators(n, c.gates, th2)).max() <= 1e-12
    s.close()


@pytest.mark.parametrize("n", [7, 8])
def test_long_clifford_runs_through_tableaus(stab, n):
    """Streamed plans apply long runs of Clifford gates as one gather through
    the run's tableau: generators, <O> and the gradient against the oracle
    (the gradient on sampled slots by the parameter shift)."""
    c = W.clifford_plus_rotations(n, 900, 10, seed=50 + n)
    s = stab.Stab(n)
    s.apply_circuit(c.gates, c.thetas)
    _, n_passes, _ = s.plan_info()
    assert n_passes < 200          # the Clifford runs did not become gate-by-gate passes
    got = layout.lib_to_paper(n, s.generators())
    ref = oracle.generators(n, c.gates, c.thetas)
    assert np.abs(got - ref).max() <= 1e-12
    obs = W.obs_chain(n) + [(0.3, "Y" * n)]
    e = s.expect(obs)
    assert abs(e - oracle.expect(n, c.gates, c.thetas, obs)) <= 1e-12 * obs_l1(obs)
    e2, g = s.grad(obs)
    assert abs(e2 - e) <= 1e-12 * obs_l1(obs)
    rot = [i for i, gt in enumerate(c.gates) if int(gt["op"]) in W.ROTATIONS]
    for gi in rot[:4]:
        want = oracle.psr_grad_gate(n, c.gates, c.thetas, obs, gi)
        assert abs(g[int(c.gates[gi]["param"])] - want) <= 1e-12 * obs_l1(obs)
    s.close()


@pytest.mark.parametrize("n", [10, 12])
def test_long_clifford_runs_large_n_vs_sparse_oracle(stab, n):
    c = W.clifford_plus_rotations(n, 1500, 8, seed=60 + n)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    obs = W.obs_chain(n)
    e = s.expect(obs)
    assert abs(e - oracle.sparse_expect(n, c.gates, c.thetas, obs)) <= 1e-12 * obs_l1(obs)
    s.close()


@pytest.mark.parametrize("n,m", [(9, 300), (10, 150)])
def test_gradient_split_wire_path(stab, n, m):
    """n = 9, 10: the split adjoint with one launch per wire pass (r forward and
    lambda backward meet mid-circuit, then both halves at once): <O> against
    the oracle and sampled slots against the oracle's parameter shift."""
    c = W.layered_ansatz(n, m, seed=70 + n)
    obs = W.obs_chain(n)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    e, g = s.grad(obs)
    s.close()
    assert abs(e - oracle.expect(n, c.gates, c.thetas, obs)) <= 1e-12 * obs_l1(obs)
    rot = [i for i, gt in enumerate(c.gates) if int(gt["op"]) in W.ROTATIONS]
    rng = np.random.default_rng(n)
    for gi in [rot[0], rot[-1]] + list(rng.choice(rot, size=2, replace=False)):
        want = oracle.psr_grad_gate(n, c.gates, c.thetas, obs, int(gi))
        assert abs(g[int(c.gates[gi]["param"])] - want) <= 1e-12 * obs_l1(obs)


def ring_pattern_circuit(n_layers, seed):
    """n = 4 layers of rotations whose wire order changes (so a layer's
    Clifford run is pulled before wire 0, 1, 2 or 3), separated by Clifford
    runs drawn from three rings in a pattern that repeats some runs and
    alternates others: the streams' repeated-pull hints are set on some
    passes and not on others, in both register layouts."""
    rng = np.random.default_rng(seed)
    rings = [[("CX", 0, 1), ("CX", 1, 2), ("CX", 2, 3), ("CX", 3, 0)],
             [("CZ", 0, 2), ("CX", 3, 1)],
             [("CX", 2, 0), ("CZ", 1, 3), ("CX", 0, 3)]]
    orders = [(0, 1, 2, 3), (2, 3, 0, 1), (1, 0, 3, 2), (3, 2, 1, 0)]
    pattern = [0, 0, 1, 0, 0, 2, 2, 1, 1, 0, 2, 0]
    gates, n_params = [], 0
    for L in range(n_layers):
        order = orders[(L // 3) % len(orders)]
        for q in order:
            for op in ("RX", "RY", "RZ"):
                gates.append((W.OPS[op], q, 0, 0, n_params))
                n_params += 1
        for op, a, b in rings[pattern[L % len(pattern)]]:
            gates.append((W.OPS[op], a, b, 0, -1))
    g = np.array(gates, dtype=W.GATE_DTYPE)
    return W.Circuit(4, g, rng.uniform(0, 2 * np.pi, n_params))


@pytest.mark.parametrize("form", ["resident", "split2", "split3"])
def test_repeated_pull_reuse_matches_oracle(stab, form):
    """A thread reuses its pull index and sign when a pass's Clifford run
    repeats the previous one (register loop at n = 4, transfer-matrix
    columns): generators, rho and <O> against the oracle on a circuit whose
    runs repeat, alternate and precede different wires."""
    from paper_2502_10685_gb300 import _lib
    import torch
    c = ring_pattern_circuit(240, seed=77)
    obs = W.random_observable(4, 7, seed=78)
    L1 = sum(abs(a) for a, _ in obs)
    name = torch.cuda.get_device_name(0)
    if form != "resident":
        stab.stab_path_store(name, 4, {"resident": 1, "resident_adjoint": 1,
                                       "gen_cut": 0.56 if form == "split2" else 0.47,
                                       "tile_limit": 1 << 17, "tuned": 1,
                                       "gen_parts": 2 if form == "split2" else 3})
    try:
        s = stab.Stab(4, kernel="resident" if form == "resident" else "auto")
        s.apply_circuit(c.gates, c.thetas)
        if form != "resident":
            assert s.split_info()[0] > 0
        gens = layout.lib_to_paper(4, s.generators())
        e = s.expect(obs)
        rho = s.density_matrix()
        s.close()
    finally:
        _lib.load().stab_path_clear()
    assert np.abs(gens - oracle.generators(4, c.gates, c.thetas)).max() <= 1e-12
    assert abs(e - oracle.expect(4, c.gates, c.thetas, obs)) <= 1e-12 * L1
    perm = _bitrev_perm(4)
    assert np.abs(rho[np.ix_(perm, perm)] - oracle.density_matrix(4, c.gates, c.thetas)).max() \
        <= 1e-12


def test_repeated_pull_reuse_in_served_slices(stab):
    """Serving slices start mid-stream, where a repeated-pull hint refers to a
    pass of an earlier slice: the kernel must walk the records then.  n = 4
    requests of the ring-pattern circuit through the iteration engine (small
    slices) equal the oracle."""
    c = ring_pattern_circuit(160, seed=79)
    obs = W.random_observable(4, 5, seed=80)
    L1 = sum(abs(a) for a, _ in obs)
    srv = stab.Server(max_active=4, engine="iterate", iter_chunks=2)
    ids = [srv.submit(c, kind, obs) for kind in ("expect", "grad", "expect")]
    res = [srv.wait(i, timeout_s=300) for i in ids]
    srv.close()
    want = oracle.expect(4, c.gates, c.thetas, obs)
    rot = [i for i, gt in enumerate(c.gates) if int(gt["op"]) in W.ROTATIONS]
    for r in res:
        assert r["status"] == 0
        assert abs(r["expect"] - want) <= 1e-12 * L1
    g = res[1]["grads"]
    for gi in (rot[1], rot[len(rot) // 2], rot[-3]):
        assert abs(g[int(c.gates[gi]["param"])] - oracle.psr_grad_gate(4, c.gates, c.thetas, obs, gi)) \
            <= 1e-12 * L1


@pytest.mark.parametrize("n,m", [(2, 6000), (3, 9000)])
def test_many_part_gradient_against_oracle(stab, n, m):
    """n <= 3, long circuits: the generators' chain cuts the plan into K >= 3
    parts (10 at n = 2, 3 at n = 3); the gradient is cut into the same parts,
    takes the pair at every cut from the chain's transfer matrices and sweeps
    all parts at once.  Sampled slots (both ends and across the parts)
    against the oracle's parameter shift, with the sweep run by the gradient
    and reused after the generators at new angles."""
    c = W.layered_ansatz(n, m, seed=630 + n)
    obs = W.random_observable(n, 3, seed=63 + n)
    l1 = sum(abs(a) for a, _ in obs)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    cut, vectors, _ = s.split_info()
    assert cut > 0 and vectors >= n + 1 + 2 * (4 ** n - 1)       # a chain of >= 3 parts
    e1, g1 = s.grad(obs)
    assert s.grad_parts() == 1 + (vectors - (n + 1)) // (4 ** n - 1)
    th2 = np.random.default_rng(640 + n).uniform(0, 2 * np.pi, c.n_params)
    s.set_params(th2)
    s.run_generators()
    e2, g2 = s.grad(obs)
    s.close()
    rot = [i for i, gt in enumerate(c.gates) if int(gt["op"]) in W.ROTATIONS]
    picks = sorted({rot[0], rot[-1]} | {rot[(len(rot) * k) // 12] for k in range(1, 12)})
    for th, e, g in ((c.thetas, e1, g1), (th2, e2, g2)):
        assert abs(e - oracle.expect(n, c.gates, th, obs)) <= 1e-12 * l1
        for gi in picks:
            want = oracle.psr_grad_gate(n, c.gates, th, obs, gi)
            assert abs(g[int(c.gates[gi]["param"])] - want) <= 1e-12 * l1, gi
