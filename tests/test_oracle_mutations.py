"""Planted mistakes in the oracle must fail its pins.

Each case compiles a copy of the oracle source with one plausible mistake
(a dropped sign, a swapped operand, a wrong digit order, a wrong CX image) on
the CPU and checks that the dense-matrix ground truth rejects it.
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import dense_ref as D

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "pauli_oracle.c")

MUTATIONS = {
    "rx_sign": ("out[2] = w[2] * c - w[3] * s;", "out[2] = w[2] * c + w[3] * s;", "RX"),
    "ry_operand": ("out[1] = w[1] * c + w[3] * s;", "out[1] = w[1] * c + w[2] * s;", "RY"),
    "h_sign": ("out[2] = -w[2];", "out[2] = w[2];", "H"),
    "s_swap": ("out[1] = -w[2]; out[2] = w[1];", "out[1] = w[2]; out[2] = -w[1];", "S"),
    "cx_sign": ('"XZ>-YY"', '"XZ>YY"', "CX"),
    "cx_image": ('"IY>ZY"', '"IY>XY"', "CX"),
    # qubit order reversed consistently (digit, 1q stride and CX strides together)
    "digit_order": ([("return (int)((idx / pow4(n - 1 - q)) % 4);",
                      "return (int)((idx / pow4(q)) % 4);"),
                     ("int64_t stride = pow4(n - 1 - q);", "int64_t stride = pow4(q);"),
                     ("int64_t sc = pow4(n - 1 - c), st = pow4(n - 1 - t);",
                      "int64_t sc = pow4(c), st = pow4(t);")], None, "RX"),
    "inverse_rotation": ("apply_row(n, q0, ROW_RZ, c, inverse ? -s : s, v);",
                         "apply_row(n, q0, ROW_RZ, c, s, v);", "RZ"),
}


def _build_mutant(name):
    old, new, _ = MUTATIONS[name]
    pairs = old if isinstance(old, list) else [(old, new)]
    src = open(SRC).read()
    for o, nw in pairs:
        assert o in src, name
        src = src.replace(o, nw, 1)
    d = tempfile.mkdtemp(prefix="orcmut_")
    path = os.path.join(d, "m.c")
    with open(path, "w") as f:
        f.write(src)
    so = os.path.join(d, "m.so")
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, path,
                           "-lm"])
    L = ctypes.CDLL(so)
    vp = ctypes.c_void_p
    L.orc_apply_gate_cs.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 2 + [ctypes.c_int, vp,
                                                                                   vp]
    return L


def _dense_mismatch(L, gate):
    n = 3
    rng = np.random.default_rng(5)
    worst = 0.0
    for trial in range(4):
        q0 = int(rng.integers(n))
        q1 = (q0 + 1) % n
        th = float(rng.uniform(0.2, 3.0))
        v = rng.normal(size=4 ** n)
        for inverse in (0, 1):
            G = D.gate_matrix(n, D.OPS[gate], q0, q1, th)
            A = D.coeffs_to_matrix(n, v)
            M = G.conj().T @ A @ G if inverse else G @ A @ G.conj().T
            want = D.matrix_to_coeffs(n, M)
            got = v.copy()
            tmp = np.empty_like(v)
            L.orc_apply_gate_cs(n, D.OPS[gate], q0, q1, math.cos(th), math.sin(th), inverse,
                                got.ctypes.data, tmp.ctypes.data)
            worst = max(worst, float(np.abs(got - want).max()))
    return worst


def test_unmutated_oracle_passes_dense_check():
    L = ctypes.CDLL(__import__("oracle").build())
    L.orc_apply_gate_cs.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 2 + [ctypes.c_int,
                                                                                   ctypes.c_void_p,
                                                                                   ctypes.c_void_p]
    for gate in ("RX", "RY", "RZ", "H", "S", "CX"):
        assert _dense_mismatch(L, gate) < 1e-12


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    L = _build_mutant(name)
    assert _dense_mismatch(L, MUTATIONS[name][2]) > 1e-3
