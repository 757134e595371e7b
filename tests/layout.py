"""Conversion between the library's coefficient layout (index = z | x << n,
bit q = qubit q) and the oracle's base-4 layout (qubit 0 most significant,
I=0 X=1 Y=2 Z=3).  Used only to compare the two in tests."""
import functools

import numpy as np


@functools.lru_cache(maxsize=16)
def lib_to_paper_index(n: int) -> np.ndarray:
    """perm[i] = base-4 index of library index i."""
    idx = np.arange(4 ** n, dtype=np.int64)
    z = idx & ((1 << n) - 1)
    x = idx >> n
    out = np.zeros_like(idx)
    for q in range(n):
        xb = (x >> q) & 1
        zb = (z >> q) & 1
        d = np.where(xb == 1, np.where(zb == 1, 2, 1), np.where(zb == 1, 3, 0))
        out += d * (4 ** (n - 1 - q))
    return out


def lib_to_paper(n: int, v: np.ndarray) -> np.ndarray:
    perm = lib_to_paper_index(n)
    out = np.empty_like(v)
    out[..., perm] = v
    return out


def paper_to_lib(n: int, v: np.ndarray) -> np.ndarray:
    perm = lib_to_paper_index(n)
    return v[..., perm]


def term_key_paper(n: int, x: int, z: int) -> int:
    """Base-4 key (qubit 0 most significant digit) of the string with masks x, z."""
    k = 0
    for q in range(n):
        xb, zb = (x >> q) & 1, (z >> q) & 1
        k = k * 4 + (2 if xb and zb else 1 if xb else 3 if zb else 0)
    return k


def terms_to_paper_dict(n: int, terms) -> dict:
    """Library term records (coeff, x, z) -> {base-4 key: coeff}."""
    return {term_key_paper(n, int(t["x"]), int(t["z"])): float(t["coeff"]) for t in terms}
