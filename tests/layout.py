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
