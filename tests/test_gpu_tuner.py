"""Path tuner on the GPU: stab_path_tune measures a valid choice for every
tuned size, AUTO contexts created afterwards run with the cached choice, and
every candidate a choice can select gives the oracle's results (generators,
<O>, gradients) -- so whichever the tuner picks on a given GPU, parity holds."""
import numpy as np
import pytest

import layout
import oracle
from paper_2502_10685_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2502_10685_gb300 import _lib, stab
    yield stab
    # forced entries must not leak into later tests: they re-tune on demand
    _lib.load().stab_path_clear()


def gpu_name():
    import torch
    return torch.cuda.get_device_name(0)


def l1(obs):
    return sum(abs(a) for a, _ in obs)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8, 9, 10])
def test_tune_gives_a_valid_choice_that_auto_contexts_use(S, n):
    c = S.stab_path_tune(0, n)
    assert c["tuned"] == 1
    assert c["resident"] in (0, 1) and c["resident_adjoint"] in (0, 1)
    assert 0.3 <= c["gen_cut"] <= 0.7 and c["tile_limit"] >= 0
    if n == 4:
        assert (c["gen_parts"], c["gen_cut"]) in (
            [(2, x) for x in (0.50, 0.53, 0.56, 0.59, 0.62)] +
            [(3, x) for x in (0.43, 0.45, 0.47, 0.49, 0.51)])
    else:
        assert c["gen_parts"] == 2
    if n >= 7:
        E = 4 ** n
        assert c["tile_limit"] in ((0, E, n * E) if n <= 9 else (1 << 17,))
    assert S.stab_path_lookup(gpu_name(), n) == c
    s = S.Stab(n)
    assert s.path_choice() == c
    s.close()
    # other kernels keep the defaults
    s = S.Stab(n, kernel="streamed")
    assert s.path_choice()["tuned"] == 0
    s.close()


@pytest.mark.parametrize("cut", [0.50, 0.62])
def test_generator_cut_candidates_match_oracle(S, cut):
    n = 4
    S.stab_path_store(gpu_name(), n, {"resident": 1, "resident_adjoint": 1, "gen_cut": cut,
                                      "tile_limit": 1 << 17, "tuned": 1})
    c = W.layered_ansatz(n, 3000, seed=4401)
    s = S.Stab(n)
    assert s.path_choice()["gen_cut"] == cut
    s.apply_circuit(c.gates, c.thetas)
    cut_pass, _, _ = s.split_info()
    n_pass = s.plan_info()[1]
    assert cut_pass == int(n_pass * cut)
    got = layout.lib_to_paper(n, s.generators())
    s.close()
    assert np.abs(got - oracle.generators(n, c.gates, c.thetas)).max() <= 1e-12


@pytest.mark.parametrize("n", [5, 6])
@pytest.mark.parametrize("resident", [0, 1])
def test_resident_and_streamed_candidates_match_oracle(S, n, resident):
    S.stab_path_store(gpu_name(), n, {"resident": resident, "resident_adjoint": resident,
                                      "gen_cut": 0.5, "tile_limit": 1 << 17, "tuned": 1})
    c = W.layered_ansatz(n, 500, seed=4500 + n)
    obs = W.obs_chain(n)
    s = S.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    assert s.plan_info()[2] == (1 if resident else 2)    # RESIDENT / STREAMED
    e, g = s.grad(obs)
    e2 = s.expect(obs)
    s.run_generators()
    gens = layout.lib_to_paper(n, s.generators())
    s.close()
    tol = 1e-12 * l1(obs)
    ref = oracle.expect(n, c.gates, c.thetas, obs)
    assert abs(e - ref) <= tol and abs(e2 - ref) <= tol
    assert np.abs(gens - oracle.generators(n, c.gates, c.thetas)).max() <= 1e-12
    rot = [i for i, gt in enumerate(c.gates) if int(gt["op"]) in W.ROTATIONS]
    for gi in (rot[3], rot[len(rot) // 2], rot[-2]):
        want = oracle.psr_grad_gate(n, c.gates, c.thetas, obs, gi)
        assert abs(g[int(c.gates[gi]["param"])] - want) <= tol


@pytest.mark.parametrize("n", [7, 8])
@pytest.mark.parametrize("tiles", [False, True])
def test_tile_limit_candidates_match_oracle(S, n, tiles):
    S.stab_path_store(gpu_name(), n, {"resident": 1, "resident_adjoint": 1, "gen_cut": 0.5,
                                      "tile_limit": (n * 4 ** n) if tiles else 0, "tuned": 1})
    c = W.layered_ansatz(n, 150, seed=4700 + n)
    obs = W.obs_chain(n)
    s = S.Stab(n)
    s.apply_circuit(c.gates, c.thetas)
    gens = layout.lib_to_paper(n, s.generators())
    e = s.expect(obs)
    s.close()
    for k in (0, n - 1):
        want = oracle.forward(n, c.gates, c.thetas, oracle.generator(n, k))
        assert np.abs(gens[k] - want).max() <= 1e-12
    assert abs(e - oracle.expect(n, c.gates, c.thetas, obs)) <= 1e-12 * l1(obs)


@pytest.mark.parametrize("m,first", [(3000, 0.43), (3001, 0.52), (60200, 0.46)])
def test_three_part_generator_split_matches_oracle(S, m, first):
    """n = 4 with the plan cut in three (a first part of `first` of the passes,
    two equal parts after it, the generators and rho_0 through the chain of
    two transfer matrices): generators, <O> and the density matrix against
    the oracle; the gradient (its own two-part adjoint) too."""
    n = 4
    S.stab_path_store(gpu_name(), n, {"resident": 1, "resident_adjoint": 1, "gen_cut": first,
                                      "tile_limit": 1 << 17, "tuned": 1, "gen_parts": 3})
    c = W.layered_ansatz(n, m, seed=4410 + m)
    obs = W.obs_chain(n)
    s = S.Stab(n)
    assert s.path_choice()["gen_parts"] == 3
    s.apply_circuit(c.gates, c.thetas)
    cut_pass, gen_units, _ = s.split_info()
    n_pass = s.plan_info()[1]
    n_mats = (gen_units - (n + 1)) // (4 ** n - 1)     # one transfer matrix per later part
    assert n_mats == 2 and cut_pass == int(n_pass * first)
    gens = layout.lib_to_paper(n, s.generators())
    e = s.expect(obs)
    rho = s.density_matrix()
    eg, g = s.grad(obs)
    s.close()
    tol = (1e-10 if m >= 60000 else 1e-12)
    assert np.abs(gens - oracle.generators(n, c.gates, c.thetas)).max() <= tol
    ref = oracle.expect(n, c.gates, c.thetas, obs)
    assert abs(e - ref) <= tol * l1(obs) and abs(eg - ref) <= tol * l1(obs)
    # library rows and columns: bit q = qubit q; the oracle's: qubit 0 most significant
    perm = [int(format(i, "0%db" % n)[::-1], 2) for i in range(2 ** n)]
    assert np.abs(rho[np.ix_(perm, perm)] - oracle.density_matrix(n, c.gates, c.thetas)).max() \
        <= tol
    assert abs(np.trace(rho) - 1) <= tol
    rot = [i for i, gt in enumerate(c.gates) if int(gt["op"]) in W.ROTATIONS]
    for gi in (rot[2], rot[len(rot) // 2]):
        want = oracle.psr_grad_gate(n, c.gates, c.thetas, obs, gi)
        assert abs(g[int(c.gates[gi]["param"])] - want) <= tol * l1(obs)


def test_three_part_choice_on_a_short_plan_keeps_two_parts(S):
    """Below three parts' minimum length the three-part choice cuts the plan
    once, at gen_cut, and the results still match the oracle."""
    n = 4
    S.stab_path_store(gpu_name(), n, {"resident": 1, "resident_adjoint": 1, "gen_cut": 0.46,
                                      "tile_limit": 1 << 17, "tuned": 1, "gen_parts": 3})
    c = W.layered_ansatz(n, 480, seed=4420)
    s = S.Stab(n)
    s.apply_circuit(c.gates, c.thetas)
    cut_pass, gen_units, _ = s.split_info()
    n_pass = s.plan_info()[1]
    n_mats = (gen_units - (n + 1)) // (4 ** n - 1)
    gens = layout.lib_to_paper(n, s.generators())
    s.close()
    assert 64 <= n_pass < 3 * 64 and n_mats == 1 and cut_pass == int(n_pass * 0.46)
    assert np.abs(gens - oracle.generators(n, c.gates, c.thetas)).max() <= 1e-12


def test_three_part_split_overlapped_async_calls_match_oracle(S):
    """The bench's step with no host synchronisation between the calls: new
    angles from device memory, the generators (context stream) and <O>
    (auxiliary stream, through the same transfer matrices) overlap; each
    step's generators and <O> match the oracle for that step's angles."""
    import torch
    n = 4
    S.stab_path_store(gpu_name(), n, {"resident": 1, "resident_adjoint": 1, "gen_cut": 0.49,
                                      "tile_limit": 1 << 17, "tuned": 1, "gen_parts": 3})
    c = W.layered_ansatz(n, 3000, seed=4430)
    obs = W.obs_chain(n)
    s = S.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    s.set_observable(obs)
    rng = np.random.default_rng(4431)
    thetas = [rng.uniform(0, 2 * np.pi, c.n_params) for _ in range(3)]
    dev = [torch.tensor(t, dtype=torch.float64, device="cuda") for t in thetas]
    outs = torch.zeros(len(dev), 8, dtype=torch.float64, device="cuda")
    gens = []
    for k, th in enumerate(dev):
        s.set_params(th)
        s.run_generators()
        s.expect_async(outs[k])
        gens.append(s.generators())           # synchronises the context stream only
    torch.cuda.synchronize()
    s.close()
    for k, th in enumerate(thetas):
        want = oracle.expect(n, c.gates, th, obs)
        assert abs(float(outs[k, 0].item()) - want) <= 1e-12 * l1(obs), k
        assert np.abs(layout.lib_to_paper(n, gens[k]) - oracle.generators(n, c.gates, th)).max() \
            <= 1e-12, k


def test_three_part_expectation_first_runs_the_sweep_itself(S):
    """n = 4, three parts: <O> asked before any generators runs the split
    sweep for the current angles itself (first part and both transfer
    matrices); after new angles it must not reuse the old sweep; the
    generators asked afterwards reuse the sweep <O> made."""
    n = 4
    S.stab_path_store(gpu_name(), n, {"resident": 1, "resident_adjoint": 1, "gen_cut": 0.49,
                                      "tile_limit": 1 << 17, "tuned": 1, "gen_parts": 3})
    c = W.layered_ansatz(n, 2400, seed=4440)
    obs = W.random_observable(n, 6, seed=4441)
    s = S.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    assert (s.split_info()[1] - (n + 1)) // (4 ** n - 1) == 2
    e1 = s.expect(obs)
    th2 = np.random.default_rng(4442).uniform(0, 2 * np.pi, c.n_params)
    s.set_params(th2)
    e2 = s.expect(obs)
    launches = s.launch_count()
    s.run_generators()              # reuses the sweep <O> made: only the products run
    ran = s.launch_count() - launches
    gens = layout.lib_to_paper(n, s.generators())
    s.close()
    assert ran == 2                 # T2 then T3 on the first-part generators
    tol = 1e-12 * l1(obs)
    assert abs(e1 - oracle.expect(n, c.gates, c.thetas, obs)) <= tol
    assert abs(e2 - oracle.expect(n, c.gates, th2, obs)) <= tol
    assert np.abs(gens - oracle.generators(n, c.gates, th2)).max() <= 1e-12


@pytest.mark.parametrize("family", ["random", "random-shared", "paper"])
def test_three_part_split_on_other_circuit_families(S, family):
    """The three-part split at n = 4 on circuits whose Clifford runs differ
    from layer to layer (random gate mixes: pulls of every length, repeated
    and not, before any wire), whose angle slots are shared by several gates,
    and on the paper's W_chain + ZXZ shape with long per-wire runs: the
    generators, <O> and the gradient against the oracle."""
    n = 4
    S.stab_path_store(gpu_name(), n, {"resident": 1, "resident_adjoint": 1, "gen_cut": 0.49,
                                      "tile_limit": 1 << 17, "tuned": 1, "gen_parts": 3})
    if family == "random":
        c = W.random_circuit(n, 4000, seed=4450)
    elif family == "random-shared":
        c = W.random_circuit(n, 4000, seed=4451, shared_params=17)
    else:
        c = W.paper_shaped_ansatz(n, 60, 20, seed=4452)
    obs = W.random_observable(n, 6, seed=4453)
    s = S.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    n_pass = s.plan_info()[1]
    if n_pass >= 3 * 64:
        assert (s.split_info()[1] - (n + 1)) // (4 ** n - 1) == 2
    s.run_generators()
    gens = layout.lib_to_paper(n, s.generators())
    e = s.expect(obs)
    eg, g = s.grad(obs)
    s.close()
    tol = 1e-12 * l1(obs)
    assert np.abs(gens - oracle.generators(n, c.gates, c.thetas)).max() <= 1e-12
    ref = oracle.expect(n, c.gates, c.thetas, obs)
    assert abs(e - ref) <= tol and abs(eg - ref) <= tol
    if family == "random-shared":
        # every slot is read by many gates: the oracle's parameter shift per slot
        want = oracle.psr_grad(n, c.gates, c.thetas, obs)
        assert np.abs(g - want).max() <= tol
    else:
        rot = [i for i, gt in enumerate(c.gates) if int(gt["op"]) in W.ROTATIONS]
        for gi in (rot[1], rot[len(rot) // 2]):
            want = oracle.psr_grad_gate(n, c.gates, c.thetas, obs, gi)
            assert abs(g[int(c.gates[gi]["param"])] - want) <= tol, (family, gi)


def with_identity_run(c, layer_gates=16, at_layer=40):
    """c with an H H pair on wire 2 inserted between the first two CNOTs of
    one layer's ring (n = 4: 12 rotation slots, then 4 CNOTs): a block of its
    own whose only wire run is the identity and holds no rotation (gradient
    plans make no pass of it, generator plans a map pass)."""
    k = layer_gates * at_layer + 13
    h = np.zeros(2, dtype=W.GATE_DTYPE)
    h["op"] = W.OPS["H"]
    h["q0"] = 2
    h["param"] = -1
    return W.Circuit(c.n, np.concatenate([c.gates[:k], h, c.gates[k:]]), c.thetas)


@pytest.mark.parametrize("parts,cut", [(3, 0.49), (2, 0.56)])
@pytest.mark.parametrize("identity_run", [False, True])
def test_gradient_cut_at_the_generators_first_part(S, parts, cut, identity_run):
    """n = 4: the gradient's cut sits where the generators' first part ends,
    and the pair at the cut comes from the generators' split sweep (rho_0
    through the first part; O backward through the later parts' transfer
    matrices, transposed) -- run by the gradient itself when no sweep was made
    for the current angles, reused when one was.  A circuit whose wire runs
    differ between the plan modes (an identity run) keeps the meet-in-the-
    middle sweep.  Both against the oracle's parameter shift."""
    n = 4
    S.stab_path_store(gpu_name(), n, {"resident": 1, "resident_adjoint": 1, "gen_cut": cut,
                                      "tile_limit": 1 << 17, "tuned": 1, "gen_parts": parts})
    c = W.layered_ansatz(n, 3200, seed=4460 + parts)
    if identity_run:
        c = with_identity_run(c)
    obs = W.random_observable(n, 5, seed=4461)
    tol = 1e-12 * l1(obs)
    rot = [i for i, gt in enumerate(c.gates) if int(gt["op"]) in W.ROTATIONS]
    picks = (rot[0], rot[len(rot) // 2 - 1], rot[len(rot) // 2 + 3], rot[-1])
    s = S.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    assert s.grad_parts() == 0
    e1, g1 = s.grad(obs)                      # no sweep for these angles yet
    # the generators' parts, or (unit sequences that differ) meet in the middle
    assert s.grad_parts() == (1 if identity_run else parts)
    th2 = np.random.default_rng(4462).uniform(0, 2 * np.pi, c.n_params)
    s.set_params(th2)
    s.run_generators()
    e2, g2 = s.grad(obs)                      # the generators' sweep, reused
    s.close()
    for th, e, g in ((c.thetas, e1, g1), (th2, e2, g2)):
        assert abs(e - oracle.expect(n, c.gates, th, obs)) <= tol
        for gi in picks:
            want = oracle.psr_grad_gate(n, c.gates, th, obs, gi)
            assert abs(g[int(c.gates[gi]["param"])] - want) <= tol, gi


@pytest.mark.parametrize("n,m", [(4, 3000), (3, 4000), (2, 4000)])
def test_density_matrix_reuses_the_sweep_a_gradient_made(S, n, m):
    """The gradient at n <= 4 runs the generators' split sweep for the current
    angles; the density matrix asked next reuses it (rho_0 through the first
    part and the parts' transfer matrices).  Both, and the generators, equal
    the oracle; after new angles nothing made for the old ones is reused."""
    c = W.layered_ansatz(n, m, seed=4470 + n)
    obs = W.random_observable(n, 4, seed=4471 + n)
    perm = [int(format(i, "0%db" % n)[::-1], 2) for i in range(2 ** n)]
    s = S.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    th2 = np.random.default_rng(4472 + n).uniform(0, 2 * np.pi, c.n_params)
    got = []
    for th in (c.thetas, th2):
        s.set_params(th)
        e, _ = s.grad(obs)
        assert s.grad_parts() >= 2
        rho = s.density_matrix()
        s.run_generators()
        gens = layout.lib_to_paper(n, s.generators())
        got.append((th, e, rho, gens))
    s.close()
    for th, e, rho, gens in got:
        assert abs(e - oracle.expect(n, c.gates, th, obs)) <= 1e-12 * l1(obs)
        assert np.abs(rho[np.ix_(perm, perm)] - oracle.density_matrix(n, c.gates, th)).max() \
            <= 1e-12
        assert np.abs(gens - oracle.generators(n, c.gates, th)).max() <= 1e-12
