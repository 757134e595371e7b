"""Stabilizer tableau (Aaronson & Gottesman, "Improved simulation of stabilizer
circuits", PRA 70, 052328 (2004)), stabilizer rows only, written from the
published update rules for CNOT, Hadamard and Phase.  Test-side ground truth
for Clifford-only circuits: generator k of |0^n> stays a single signed Pauli
string, row k of this tableau.  (x, z) = (1, 1) denotes Y, as in that paper.
"""
from __future__ import annotations

import numpy as np


class Tableau:
    def __init__(self, n: int):
        self.n = n
        self.x = np.zeros((n, n), dtype=bool)
        self.z = np.eye(n, dtype=bool)      # row k = Z_k
        self.r = np.zeros(n, dtype=bool)

    def h(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.x[:, a], self.z[:, a] = self.z[:, a].copy(), self.x[:, a].copy()

    def s(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.z[:, a] ^= self.x[:, a]

    def cnot(self, a, b):
        self.r ^= self.x[:, a] & self.z[:, b] & ~(self.x[:, b] ^ self.z[:, a])
        self.x[:, b] ^= self.x[:, a]
        self.z[:, a] ^= self.z[:, b]

    def row(self, k):
        """(sign, string) of stabilizer row k."""
        letters = []
        for q in range(self.n):
            xb, zb = self.x[k, q], self.z[k, q]
            letters.append("Y" if xb and zb else "X" if xb else "Z" if zb else "I")
        return (-1 if self.r[k] else 1), "".join(letters)
