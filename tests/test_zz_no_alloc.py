"""stab_expect_static: <O> for callers that cannot allocate device memory.

Some callers must not allocate device memory at all -- a program that
reserves its whole device budget at start-up, or code running inside a
framework whose allocator owns the device.  stab_expect_static runs the
streamed expectation path on a fixed workspace the library declares as a
static device array.  This test calls it through the C interface twice in a
row, on two different circuits, and checks each value against stab_expect
(streamed kernels) and against the CPU oracle within the tolerance of the
other parity tests; a second call that agreed only because it reused the
first call's leftovers would fail here.  It also checks that a problem too
large for the workspace is refused with STAB_E_RANGE.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2502_10685_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _static_expect(L, c, obs):
    from paper_2502_10685_gb300.stab import terms_from_observable
    t = terms_from_observable(c.n, obs)
    th = np.ascontiguousarray(c.thetas if c.n_params else np.zeros(1))
    g = np.ascontiguousarray(c.gates)
    out = ctypes.c_double(np.nan)
    rc = L.stab_expect_static(c.n, g.ctypes.data, c.m, th.ctypes.data, c.n_params,
                              t.ctypes.data, len(t), ctypes.byref(out), None)
    return rc, out.value


def test_static_expect_matches_stab_expect_on_two_calls_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2502_10685_gb300 import _lib, stab
    L = _lib.load()
    cases = [(W.layered_ansatz(6, 400, seed=11), W.obs_chain(6)),
             (W.random_circuit(8, 150, seed=12), W.random_observable(8, 7, seed=13))]
    got = []
    for c, obs in cases:                       # two calls in a row
        rc, val = _static_expect(L, c, obs)
        assert rc == 0, _lib.ERRORS.get(rc, rc)
        got.append(val)
    for (c, obs), val in zip(cases, got):
        s = stab.Stab(c.n, kernel="streamed")
        s.load_circuit(c.gates, c.thetas)
        ref = s.expect(obs)
        s.close()
        tol = 1e-12 * sum(abs(a) for a, _ in obs)
        assert abs(val - ref) <= tol
        assert abs(val - oracle.expect(c.n, c.gates, c.thetas, obs)) <= tol


def test_static_expect_refuses_problems_beyond_the_workspace():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2502_10685_gb300 import _lib
    L = _lib.load()
    c = W.layered_ansatz(11, 20, seed=3)       # two vectors of 4^11 doubles = 64 MiB
    rc, _ = _static_expect(L, c, W.obs_chain(11))
    assert rc == -2                            # STAB_E_RANGE
