"""ctypes front end of the plain FP64 CPU oracle (``pauli_oracle.c``, dense
4^n vectors, and ``sparse_oracle.c``, lists of (coefficient, string) terms).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference legs of ``bench.py`` use it; the CUDA library never
does.  Vectors here use the paper's base-4 encoding (Sec. III-B): qubit 0 is
the most significant digit and I, X, Y, Z are 0, 1, 2, 3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("pauli_oracle.c", "sparse_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GATE_DTYPE = np.dtype([("op", "u1"), ("q0", "u1"), ("q1", "u1"), ("flags", "u1"),
                       ("param", "<i4")])

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction)."""
    stale = not os.path.exists(_LIB) or any(
        os.path.getmtime(_LIB) < os.path.getmtime(f) for f in _SRCS)
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64, c_int, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            L.orc_string_to_index.restype = i64
            L.orc_string_to_index.argtypes = [ctypes.c_char_p]
            L.orc_index_to_string.argtypes = [c_int, i64, ctypes.c_char_p]
            L.orc_apply_gate_cs.argtypes = [c_int, c_int, c_int, c_int, ctypes.c_double,
                                            ctypes.c_double, c_int, vp, vp]
            for name in ("orc_forward", "orc_backward", "orc_generators"):
                getattr(L, name).argtypes = [c_int, i64, vp, vp, i64, vp]
                getattr(L, name).restype = c_int
            L.orc_validate.argtypes = [c_int, i64, vp, i64]
            L.orc_init_generator.argtypes = [c_int, c_int, vp]
            L.orc_sum_xfree.argtypes = [c_int, vp]
            L.orc_sum_xfree.restype = ctypes.c_double
            L.orc_expect.argtypes = [c_int, i64, vp, vp, i64, vp, vp]
            L.orc_psr_grad.argtypes = [c_int, i64, vp, vp, i64, vp, vp]
            L.orc_psr_grad_gate.argtypes = [c_int, i64, vp, vp, i64, vp, i64, vp]
            L.orc_expand.argtypes = [c_int, c_int, vp, vp]
            L.orc_map_noncx.argtypes = [c_int, ctypes.c_double, ctypes.c_double, vp, vp]
            L.orc_density_matrix.argtypes = [c_int, i64, vp, vp, i64, vp, vp]
            L.orc_sparse_propagate.argtypes = [c_int, i64, vp, vp, i64, c_int, i64, vp, vp,
                                               i64, vp, vp, vp]
            L.orc_sparse_sum_xfree.argtypes = [c_int, i64, vp, vp]
            L.orc_sparse_sum_xfree.restype = ctypes.c_double
            L.orc_sparse_expect.argtypes = [c_int, i64, vp, vp, i64, i64, vp, vp, vp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _gates(g) -> np.ndarray:
    g = np.ascontiguousarray(g)
    if g.dtype.itemsize != 8 or g.dtype.names is None:
        raise TypeError("gate records must be the 8-byte {op,q0,q1,flags,param} layout")
    return g.view(GATE_DTYPE)


def _thetas(t) -> np.ndarray:
    t = np.ascontiguousarray(t, dtype=np.float64)
    if t.size == 0:
        t = np.zeros(1)
    return t


def string_to_index(s: str) -> int:
    return int(lib().orc_string_to_index(s.encode()))


def index_to_string(n: int, idx: int) -> str:
    buf = ctypes.create_string_buffer(n + 1)
    lib().orc_index_to_string(n, idx, buf)
    return buf.value.decode()


def dense_observable(n: int, terms) -> np.ndarray:
    """Observable terms [(coeff, string)] -> dense base-4 coefficient vector."""
    v = np.zeros(4 ** n)
    for c, s in terms:
        if len(s) != n:
            raise ValueError("observable string length must equal n")
        i = string_to_index(s)
        if i < 0:
            raise ValueError("bad Pauli letter in %r" % s)
        v[i] += c
    return v


def generator(n: int, k: int) -> np.ndarray:
    v = np.zeros(4 ** n)
    lib().orc_init_generator(n, k, _p(v))
    return v


def apply_gate(n: int, op: int, q0: int, q1: int, v: np.ndarray, c: float = 1.0,
               s: float = 0.0, inverse: bool = False) -> np.ndarray:
    """Conjugate the dense vector by one gate, with (cos, sin) given directly."""
    v = np.ascontiguousarray(v, dtype=np.float64).copy()
    tmp = np.empty_like(v)
    lib().orc_apply_gate_cs(n, op, q0, q1, c, s, int(inverse), _p(v), _p(tmp))
    return v


def forward(n: int, gates, thetas, v: np.ndarray) -> np.ndarray:
    g, t = _gates(gates), _thetas(thetas)
    v = np.ascontiguousarray(v, dtype=np.float64).copy()
    rc = lib().orc_forward(n, g.shape[0], _p(g), _p(t), len(np.atleast_1d(thetas)), _p(v))
    if rc != 0:
        raise ValueError("oracle: invalid circuit")
    return v


def backward(n: int, gates, thetas, v: np.ndarray) -> np.ndarray:
    g, t = _gates(gates), _thetas(thetas)
    v = np.ascontiguousarray(v, dtype=np.float64).copy()
    rc = lib().orc_backward(n, g.shape[0], _p(g), _p(t), len(np.atleast_1d(thetas)), _p(v))
    if rc != 0:
        raise ValueError("oracle: invalid circuit")
    return v


def generators(n: int, gates, thetas) -> np.ndarray:
    """The n evolved generators U Z_k U^dagger, shape (n, 4^n), base-4 layout."""
    g, t = _gates(gates), _thetas(thetas)
    out = np.empty((n, 4 ** n))
    rc = lib().orc_generators(n, g.shape[0], _p(g), _p(t), len(np.atleast_1d(thetas)), _p(out))
    if rc != 0:
        raise ValueError("oracle: invalid circuit")
    return out


def sum_xfree(n: int, v: np.ndarray) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(lib().orc_sum_xfree(n, _p(v)))


def expect(n: int, gates, thetas, terms) -> float:
    """<0^n| U^dagger O U |0^n> by backward propagation of O."""
    g, t = _gates(gates), _thetas(thetas)
    O = dense_observable(n, terms)
    out = ctypes.c_double()
    rc = lib().orc_expect(n, g.shape[0], _p(g), _p(t), len(np.atleast_1d(thetas)), _p(O),
                          ctypes.byref(out))
    if rc != 0:
        raise ValueError("oracle: invalid circuit")
    return out.value


def psr_grad(n: int, gates, thetas, terms) -> np.ndarray:
    g, t = _gates(gates), _thetas(thetas)
    n_params = len(np.atleast_1d(thetas))
    O = dense_observable(n, terms)
    out = np.zeros(max(n_params, 1))
    rc = lib().orc_psr_grad(n, g.shape[0], _p(g), _p(t), n_params, _p(O), _p(out))
    if rc != 0:
        raise ValueError("oracle: invalid circuit")
    return out[:n_params]


def psr_grad_gate(n: int, gates, thetas, terms, gate_index: int) -> float:
    g, t = _gates(gates), _thetas(thetas)
    O = dense_observable(n, terms)
    out = ctypes.c_double()
    rc = lib().orc_psr_grad_gate(n, g.shape[0], _p(g), _p(t), len(np.atleast_1d(thetas)),
                                 _p(O), gate_index, ctypes.byref(out))
    if rc != 0:
        raise ValueError("oracle: gate is not a rotation")
    return out.value


def expand(weights: np.ndarray) -> np.ndarray:
    """Eq. (5) flatten+reduce: weights (terms, n, 4) -> dense 4^n vector."""
    W = np.ascontiguousarray(weights, dtype=np.float64)
    T, n, four = W.shape
    assert four == 4
    out = np.empty(4 ** n)
    lib().orc_expand(n, T, _p(W), _p(out))
    return out


def map_noncx(op: int, w, c: float = 1.0, s: float = 0.0) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty(4)
    lib().orc_map_noncx(op, c, s, _p(w), _p(out))
    return out


def density_matrix(n: int, gates, thetas) -> np.ndarray:
    """rho = |psi><psi| of U|0^n> decoded from the Pauli coefficients (Sec. III-D,
    Eq. (3)); complex (2^n, 2^n), qubit 0 the most significant bit."""
    g, t = _gates(gates), _thetas(thetas)
    D = 2 ** n
    re = np.empty((D, D))
    im = np.empty((D, D))
    rc = lib().orc_density_matrix(n, g.shape[0], _p(g), _p(t), len(np.atleast_1d(thetas)),
                                  _p(re), _p(im))
    if rc != 0:
        raise ValueError("oracle: invalid circuit")
    return re + 1j * im


# ---------------------------------------------------------------- sparse lists

def sparse_terms(n: int, terms):
    """[(coeff, string)] -> (keys uint64, coeffs float64) in the base-4 encoding
    (qubit 0 the most significant digit); works for n <= 32."""
    keys = np.zeros(len(terms), dtype=np.uint64)
    vals = np.zeros(len(terms))
    for i, (c, s) in enumerate(terms):
        if len(s) != n:
            raise ValueError("observable string length must equal n")
        k = 0
        for ch in s:
            d = "IXYZ".find(ch)
            if d < 0:
                raise ValueError("bad Pauli letter in %r" % s)
            k = k * 4 + d
        keys[i] = k
        vals[i] = c
    return keys, vals


def sparse_propagate(n: int, gates, thetas, keys, vals, backward: bool = False,
                     cap: int = 1 << 22):
    """Propagate a term list through the circuit (forward: U P U^dagger; backward:
    U^dagger P U).  Returns (keys, coeffs) sorted by key, exact zeros dropped."""
    g, t = _gates(gates), _thetas(thetas)
    k_in = np.ascontiguousarray(keys, dtype=np.uint64)
    v_in = np.ascontiguousarray(vals, dtype=np.float64)
    k_out = np.zeros(max(cap, 1), dtype=np.uint64)
    v_out = np.zeros(max(cap, 1))
    n_out = ctypes.c_int64()
    rc = lib().orc_sparse_propagate(n, g.shape[0], _p(g), _p(t), len(np.atleast_1d(thetas)),
                                    int(backward), k_in.size, _p(k_in), _p(v_in), cap,
                                    _p(k_out), _p(v_out), ctypes.byref(n_out))
    if rc == -2:
        raise OverflowError("oracle: %d terms exceed cap %d" % (n_out.value, cap))
    if rc != 0:
        raise ValueError("oracle: invalid circuit or input (%d)" % rc)
    return k_out[:n_out.value].copy(), v_out[:n_out.value].copy()


def sparse_generator(n: int, gates, thetas, k: int):
    """U Z_k U^dagger as a term list (keys, coeffs)."""
    keys, vals = sparse_terms(n, [(1.0, "I" * k + "Z" + "I" * (n - k - 1))])
    return sparse_propagate(n, gates, thetas, keys, vals, backward=False)


def sparse_sum_xfree(n: int, keys, vals) -> float:
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    v = np.ascontiguousarray(vals, dtype=np.float64)
    return float(lib().orc_sparse_sum_xfree(n, k.size, _p(k), _p(v)))


def sparse_expect(n: int, gates, thetas, terms) -> float:
    """<0^n| U^dagger O U |0^n> on term lists (any n <= 32)."""
    g, t = _gates(gates), _thetas(thetas)
    k, v = sparse_terms(n, terms)
    out = ctypes.c_double()
    rc = lib().orc_sparse_expect(n, g.shape[0], _p(g), _p(t), len(np.atleast_1d(thetas)),
                                 k.size, _p(k), _p(v), ctypes.byref(out))
    if rc != 0:
        raise ValueError("oracle: invalid circuit or input (%d)" % rc)
    return out.value
