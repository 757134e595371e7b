"""The C library loads without a GPU and exports every symbol include/stab.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(stab_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_core_entry_points():
    names = declared_functions()
    for core in ("stab_create", "stab_apply_circuit", "stab_get_generators", "stab_expect",
                 "stab_grad", "stab_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol():
    from paper_2502_10685_gb300 import _lib
    L = _lib.load()
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, missing


def test_host_only_calls():
    from paper_2502_10685_gb300 import _lib, stab
    L = _lib.load()
    assert L.stab_version() == 1
    assert L.stab_error_string(-5) == b"non-finite angle or coefficient"
    o = stab.stab_default_opts()
    assert o.device == -1 and o.fuse == 1 and o.kernel == 0


def test_chunked_planner_equals_sequential():
    # host-only: long gate lists are planned in parallel chunks; the plan and
    # its instruction streams must be byte-identical to the sequential ones,
    # and streams built as two pieces at once must apply the same pulls and
    # passes in the same order as the one-piece streams; a pass header is
    # flagged as a repeated pull exactly when its pull records equal the
    # previous pull pass's
    import numpy as np
    from paper_2502_10685_gb300 import _lib, workloads as W
    L = _lib.load()
    cases = [W.layered_ansatz(4, 60200, seed=1002), W.layered_ansatz(8, 20000, seed=3),
             W.random_circuit(5, 30000, seed=11), W.random_circuit(3, 20000, seed=12,
                                                                     shared_params=9),
             W.paper_shaped_ansatz(4, 50, 100, seed=13)]
    for c in cases:
        g = np.ascontiguousarray(c.gates)
        for mode in range(4):
            rc = L.stab_selftest_plan(c.n, g.ctypes.data, len(g), c.n_params, mode)
            assert rc == 0, (c.n, len(g), mode, rc)
    assert L.stab_selftest_plan(2, g.ctypes.data, len(g), c.n_params, 7) != 0


def test_server_options_rejected_on_the_host():
    # host-only: malformed server options are refused before any device call
    import ctypes
    from paper_2502_10685_gb300 import _lib
    L = _lib.load()
    for field, value in (("policy", 7), ("engine", 5), ("iter_chunks", -1),
                         ("iter_smem_kb", 201), ("iter_max_n", 9), ("iter_max_n", -1),
                         ("iter_slice_us", float("nan")), ("iter_slice_us", 2e6)):
        o = _lib.StabServerOpts()
        setattr(o, field, value)
        h = ctypes.c_void_p()
        assert L.stab_server_create(ctypes.byref(o), ctypes.byref(h)) == -1, field
        assert not h.value
    # only one of the two allocator hooks
    o = _lib.StabServerOpts()
    keep = _lib.ALLOC_FN(lambda n, s, u: None)
    o.alloc = keep
    h = ctypes.c_void_p()
    assert L.stab_server_create(ctypes.byref(o), ctypes.byref(h)) == -1


def split_sweep_bytes(n):
    # n <= 4: the transfer matrices, n + 1 first-part vectors, two pair vectors per matrix
    if n > 4:
        return 0
    E = 4 ** n
    mats = 2 if n == 4 else max(1, min(49, 160 // (E - 1)))
    return 8 * (mats * E * E + (n + 1 + 2 * mats) * E)


def test_request_footprint_counts_the_split_sweep_vectors():
    # host-only: max(n, 12) vectors of 4^n doubles for a gradient (half sweeps
    # and two (lambda, rho) pairs with spares), max(n, 4) for an expectation,
    # plus 96 B per gate, plus the split sweep's transfer matrices at n <= 4
    import ctypes
    from paper_2502_10685_gb300 import _lib
    L = _lib.load()
    r = _lib.StabRequest()
    r.n, r.m = 3, 1000
    r.kind = 0
    assert L.stab_request_footprint(ctypes.byref(r)) == \
        4 * 8 * 4 ** 3 + 96 * 1000 + split_sweep_bytes(3)
    # gradients at n <= 5 add the resident sweep's per-thread dot shares (one
    # row of its CTA's threads per gate, as a bound on the rotations)
    r.kind = 1
    for n, threads in ((3, 32), (4, 64), (5, 256)):
        r.n = n
        assert L.stab_request_footprint(ctypes.byref(r)) == \
            12 * 8 * 4 ** n + 96 * 1000 + 8 * 1000 * threads + split_sweep_bytes(n)
    r.n = 6
    assert L.stab_request_footprint(ctypes.byref(r)) == 12 * 8 * 4 ** 6 + 96 * 1000
    r.kind = 0
    r.n = 8
    assert L.stab_request_footprint(ctypes.byref(r)) == 8 * 8 * 4 ** 8 + 96 * 1000
    r.kind = 1
    assert L.stab_request_footprint(ctypes.byref(r)) >= 12 * 8 * 4 ** 8 + 96 * 1000
    r.n, r.kind = 12, 0
    assert L.stab_request_footprint(ctypes.byref(r)) == 12 * 8 * 4 ** 12 + 96 * 1000
    r.n = 13
    assert L.stab_request_footprint(ctypes.byref(r)) == 0


def test_fp64_probe_rejects_bad_arguments_on_the_host():
    # host-only: argument checks come before any device call
    import ctypes
    from paper_2502_10685_gb300 import _lib
    L = _lib.load()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    assert L.stab_probe_fp64(2, 1024, ctypes.byref(tf), ctypes.byref(ms)) == -1
    assert L.stab_probe_fp64(0, 1024, None, ctypes.byref(ms)) == -1
    assert L.stab_probe_fp64(0, 0, ctypes.byref(tf), ctypes.byref(ms)) == -2
    assert L.stab_probe_fp64(1, (1 << 30) + 1, ctypes.byref(tf), ctypes.byref(ms)) == -2


def test_grad_parts_rejects_null_on_the_host():
    # host-only: argument checks come before any device call
    import ctypes
    from paper_2502_10685_gb300 import _lib
    L = _lib.load()
    k = ctypes.c_int32()
    assert L.stab_grad_parts(None, ctypes.byref(k)) == -1


def test_pass_probe_rejects_bad_arguments_on_the_host():
    # host-only: argument checks come before any device call
    import ctypes
    from paper_2502_10685_gb300 import _lib
    L = _lib.load()
    c = ctypes.c_double()
    for pattern, threads in ((5, 256), (-1, 256), (0, 64), (0, 512), (3, 256)):
        assert L.stab_probe_pass(pattern, threads, 1024, ctypes.byref(c)) == -1
    assert L.stab_probe_pass(0, 256, 1024, None) == -1
    for passes in (0, 2, 1026, (1 << 24) + 4):
        assert L.stab_probe_pass(0, 256, passes, ctypes.byref(c)) == -2


def test_gradient_cut_alignment_on_the_host():
    # host-only: every generator-plan unit boundary maps to a gradient-plan
    # pass with the same rotations and two-qubit gates before it; a circuit
    # with a wire run that is the identity (no pass in the gradient plan) is
    # refused, and only such a circuit
    import ctypes
    import numpy as np
    from paper_2502_10685_gb300 import _lib, workloads as W
    L = _lib.load()

    def check(c):
        g = np.ascontiguousarray(c.gates)
        out = ctypes.c_int64()
        rc = L.stab_selftest_align(c.n, g.ctypes.data, len(g), c.n_params, ctypes.byref(out))
        assert rc == 0, (c.n, len(g), rc)
        return out.value

    for c in (W.layered_ansatz(4, 3000, seed=1), W.layered_ansatz(3, 2000, seed=2),
              W.layered_ansatz(2, 1500, seed=3), W.layered_ansatz(5, 800, seed=4),
              W.paper_shaped_ansatz(4, 20, 30, seed=5)):
        assert check(c) > 0
    for seed in range(6):
        check(W.random_circuit(4, 1500, seed=100 + seed))
        check(W.random_circuit(3, 1500, seed=200 + seed, shared_params=7))
    # a wire run longer than one pass takes (16,384 gates): two consecutive
    # passes on one wire in the generator plan, many in the gradient plan --
    # still one unit in both
    rng = np.random.default_rng(7)
    layer = W.layered_ansatz(2, 400, seed=7)
    long_run = np.zeros(20000, dtype=W.GATE_DTYPE)
    long_run["op"] = rng.choice([W.OPS["RX"], W.OPS["RY"], W.OPS["RZ"]], size=20000)
    long_run["q0"] = 0
    long_run["param"] = np.arange(20000) + layer.n_params
    cx = np.zeros(1, dtype=W.GATE_DTYPE)
    cx["op"] = W.OPS["CX"]
    cx["q0"], cx["q1"], cx["param"] = 0, 1, -1
    gl = np.concatenate([layer.gates, cx, long_run, cx, layer.gates])
    th = np.concatenate([layer.thetas, rng.uniform(0, 6.28, 20000)])
    assert check(W.Circuit(2, gl, th)) > 0
    # an H H pair between two CNOTs of a ring: a block whose one wire run is
    # the identity -- the aligner must refuse (0 passes aligned)
    c = W.layered_ansatz(4, 1600, seed=6)
    h = np.zeros(2, dtype=W.GATE_DTYPE)
    h["op"] = W.OPS["H"]
    h["q0"] = 2
    h["param"] = -1
    k = 16 * 30 + 13
    c2 = W.Circuit(4, np.concatenate([c.gates[:k], h, c.gates[k:]]), c.thetas)
    assert check(c2) == 0
