"""Uniform dyadic (1D) and quad (2D) trees over the n^d grid, in Morton order.

Section 2 defines the trees T_X and T_Omega by recursive dyadic partitioning of X and Omega;
section 3 uses the same partition of Omega for the hierarchical matrix of K*K.  Both grids have
the same shape, so one tree object serves both.

Node ids: at level l there are beta^l nodes (beta = 2^d); node i has children beta*i + c,
c = 0..beta-1.  For d = 2 the node id is the Morton code of its cell coordinates (a1, a2), bit t
of a1 going to bit 2t and bit t of a2 to bit 2t+1.  Every node's points are a contiguous range of
the Morton permutation ``perm`` of the grid, so a node's points are the concatenation of its
children's points.  Grid points use the linear index i1 + n*i2 (the C ABI's natural order).
"""

from __future__ import annotations

import numpy as np


def morton_encode(a1: np.ndarray, a2: np.ndarray, bits: int) -> np.ndarray:
    a1 = np.asarray(a1, dtype=np.int64)
    a2 = np.asarray(a2, dtype=np.int64)
    code = np.zeros(np.broadcast(a1, a2).shape, dtype=np.int64)
    for t in range(bits):
        code |= ((a1 >> t) & 1) << (2 * t)
        code |= ((a2 >> t) & 1) << (2 * t + 1)
    return code


def morton_decode(code: np.ndarray, bits: int):
    code = np.asarray(code, dtype=np.int64)
    a1 = np.zeros_like(code)
    a2 = np.zeros_like(code)
    for t in range(bits):
        a1 |= ((code >> (2 * t)) & 1) << t
        a2 |= ((code >> (2 * t + 1)) & 1) << t
    return a1, a2


class Tree:
    """Complete tree of depth `depth` over an n^d grid (n a power of two)."""

    def __init__(self, d: int, n: int, depth: int):
        if n & (n - 1):
            raise ValueError("n must be a power of two")
        self.d, self.n, self.depth = d, n, depth
        self.N = n ** d
        self.beta = 2 ** d
        if self.N % (self.beta ** depth):
            raise ValueError("tree deeper than the grid")
        self.bits = int(round(np.log2(n)))
        if d == 1:
            self.perm = np.arange(n, dtype=np.int64)
        else:
            codes = np.arange(self.N, dtype=np.int64)
            i1, i2 = morton_decode(codes, self.bits)
            self.perm = i1 + n * i2  # perm[morton position] = natural index
        self.pos = np.empty(self.N, dtype=np.int64)  # natural index -> Morton position
        self.pos[self.perm] = np.arange(self.N)

    def count(self, level: int) -> int:
        return self.beta ** level

    def size(self, level: int) -> int:
        """Points per node at `level`."""
        return self.N // self.beta ** level

    def points(self, level: int, node: int) -> np.ndarray:
        s = self.size(level)
        return self.perm[node * s:(node + 1) * s]

    def cell_coords(self, level: int, node: np.ndarray):
        """Cell coordinates (a1[, a2]) of nodes at `level` (2D: Morton decode)."""
        node = np.asarray(node, dtype=np.int64)
        if self.d == 1:
            return (node,)
        return morton_decode(node, level)

    def cell_id(self, level: int, a1, a2=None):
        if self.d == 1:
            return np.asarray(a1, dtype=np.int64)
        return morton_encode(a1, a2, level)
