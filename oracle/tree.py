"""HODLR partition tree (Sec. 3.2 of the paper; SI example of a 2-level tree).

The sorted index range [0, n) is split recursively into two halves; a node
[s, e) splits at h = s + floor((e - s) / 2).  The recursion stops when every
node has at most B indices (B = maximum block size, Algorithm 1 inputs).  All
leaves sit at the same depth L, the smallest depth at which ceil(n / 2**L) <= B.
Level l holds 2**l nodes; node i of level l covers [bounds[l][i], bounds[l][i+1]).
"""
from __future__ import annotations

import numpy as np


def num_levels(n: int, B: int) -> int:
    if n < 1 or B < 1:
        raise ValueError("n and B must be >= 1")
    L = 0
    while -(-n // (1 << L)) > B:
        L += 1
    return L


class Tree:
    def __init__(self, n: int, B: int):
        self.n, self.B = n, B
        self.L = num_levels(n, B)
        self.bounds = [np.array([0, n], dtype=np.int64)]
        for _ in range(self.L):
            prev = self.bounds[-1]
            nxt = [0]
            for i in range(len(prev) - 1):
                s, e = int(prev[i]), int(prev[i + 1])
                nxt += [s + (e - s) // 2, e]
            self.bounds.append(np.array(nxt, dtype=np.int64))

    def node(self, lvl: int, i: int):
        """(s, h, e): node range [s, e) and the split point h between its children."""
        s, e = int(self.bounds[lvl][i]), int(self.bounds[lvl][i + 1])
        return s, s + (e - s) // 2, e

    def leaves(self):
        b = self.bounds[self.L]
        return [(int(b[i]), int(b[i + 1])) for i in range(len(b) - 1)]
