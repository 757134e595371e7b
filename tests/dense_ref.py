"""Dense-matrix ground truth for small n (test-side, independent of the oracle).

Gates are built as explicit 2^n x 2^n complex matrices from their textbook
definitions: H = (X+Z)/sqrt2, S = diag(1, i), R_s(theta) = exp(-i theta s / 2),
CX(c->t) = |0><0|_c + |1><1|_c X_t, CZ = diag(1,1,1,-1) on (a, b).  Tensor
factor j of a Pauli string is qubit j (qubit 0 leftmost), the order of the
paper's strings.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = {"I": I2, "X": PX, "Y": PY, "Z": PZ}
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)

OPS = {"H": 0, "S": 1, "SDG": 2, "X": 3, "Y": 4, "Z": 5, "CX": 6, "CZ": 7,
       "RX": 8, "RY": 9, "RZ": 10}


def kron_all(mats):
    out = np.array([[1.0 + 0j]])
    for m in mats:
        out = np.kron(out, m)
    return out


def pauli_matrix(s: str) -> np.ndarray:
    return kron_all([PAULI[ch] for ch in s])


def rot(sigma: np.ndarray, theta: float) -> np.ndarray:
    return math.cos(theta / 2) * I2 - 1j * math.sin(theta / 2) * sigma


def one_qubit_matrix(op: int, theta: float = 0.0) -> np.ndarray:
    if op == OPS["H"]:
        return (PX + PZ) / math.sqrt(2)
    if op == OPS["S"]:
        return np.diag([1, 1j])
    if op == OPS["SDG"]:
        return np.diag([1, -1j])
    if op == OPS["X"]:
        return PX
    if op == OPS["Y"]:
        return PY
    if op == OPS["Z"]:
        return PZ
    if op == OPS["RX"]:
        return rot(PX, theta)
    if op == OPS["RY"]:
        return rot(PY, theta)
    if op == OPS["RZ"]:
        return rot(PZ, theta)
    raise ValueError(op)


def gate_matrix(n: int, op: int, q0: int, q1: int = 0, theta: float = 0.0) -> np.ndarray:
    if op == OPS["CX"]:
        a = [I2] * n
        b = [I2] * n
        a[q0] = P0
        b[q0] = P1
        b[q1] = PX
        return kron_all(a) + kron_all(b)
    if op == OPS["CZ"]:
        a = [I2] * n
        b = [I2] * n
        a[q0] = P0
        b[q0] = P1
        b[q1] = PZ
        return kron_all(a) + kron_all(b)
    mats = [I2] * n
    mats[q0] = one_qubit_matrix(op, theta)
    return kron_all(mats)


def circuit_unitary(n: int, gates, thetas) -> np.ndarray:
    U = np.eye(2 ** n, dtype=complex)
    for g in gates:
        th = float(thetas[g["param"]]) if g["op"] >= OPS["RX"] else 0.0
        U = gate_matrix(n, int(g["op"]), int(g["q0"]), int(g["q1"]), th) @ U
    return U


def all_strings(n: int):
    return ["".join(p) for p in itertools.product("IXYZ", repeat=n)]


def coeffs_to_matrix(n: int, v: np.ndarray) -> np.ndarray:
    """sum_P v_P P with P in base-4 order (qubit 0 most significant)."""
    A = np.zeros((2 ** n, 2 ** n), dtype=complex)
    for i, s in enumerate(all_strings(n)):
        if v[i] != 0:
            A += v[i] * pauli_matrix(s)
    return A


def matrix_to_coeffs(n: int, A: np.ndarray) -> np.ndarray:
    """c_P = Tr(P A) / 2^n, base-4 order; asserts the result is real."""
    out = np.zeros(4 ** n, dtype=complex)
    for i, s in enumerate(all_strings(n)):
        out[i] = np.trace(pauli_matrix(s) @ A) / 2 ** n
    assert np.max(np.abs(out.imag)) < 1e-12
    return out.real


def statevector_expect(n: int, gates, thetas, terms) -> float:
    """<psi|O|psi> with psi = U|0^n>, gate by gate on a 2^n state vector."""
    psi = np.zeros(2 ** n, dtype=complex)
    psi[0] = 1.0
    for g in gates:
        op, q0, q1 = int(g["op"]), int(g["q0"]), int(g["q1"])
        th = float(thetas[g["param"]]) if op >= OPS["RX"] else 0.0
        t = psi.reshape([2] * n)
        if op in (OPS["CX"], OPS["CZ"]):
            M = np.zeros((4, 4), dtype=complex)
            M[0, 0] = M[1, 1] = 1
            if op == OPS["CX"]:
                M[2, 3] = M[3, 2] = 1
            else:
                M[2, 2] = 1
                M[3, 3] = -1
            t = np.moveaxis(t, (q0, q1), (0, 1))
            shp = t.shape
            t = (M @ t.reshape(4, -1)).reshape(shp)
            t = np.moveaxis(t, (0, 1), (q0, q1))
        else:
            M = one_qubit_matrix(op, th)
            t = np.moveaxis(t, q0, 0)
            shp = t.shape
            t = (M @ t.reshape(2, -1)).reshape(shp)
            t = np.moveaxis(t, 0, q0)
        psi = t.reshape(-1)
    val = 0.0
    for c, s in terms:
        val += c * np.vdot(psi, _apply_pauli_string(n, s, psi)).real
    return val


def _apply_pauli_string(n: int, s: str, psi: np.ndarray) -> np.ndarray:
    t = psi.reshape([2] * n)
    for q, ch in enumerate(s):
        if ch == "I":
            continue
        t = np.moveaxis(t, q, 0)
        shp = t.shape
        t = (PAULI[ch] @ t.reshape(2, -1)).reshape(shp)
        t = np.moveaxis(t, 0, q)
    return t.reshape(-1)
