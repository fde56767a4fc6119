"""Sparse stage objects produced by the builders and consumed by the packer.

Every factor of the method is stored as a *stage*: a list of small dense complex blocks, each
with the index list it reads (``inp``) and the index list it writes (``out``).

* MAP stage (butterfly factors, section 2): y = S x with y a new vector of length ``out_len``.
  Every output index is written by exactly one block row and every input index is read by at
  most one block column, so S and S* are both "block diagonal up to permutations".
* INPLACE stage (HIF factors, section 4, and the root): x[I_b] <- M_b x[I_b] for disjoint index
  sets I_b; the identity elsewhere.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

KIND_MAP = 0
KIND_INPLACE = 1

ROLE_BF = 0
ROLE_HIF_CELL = 1
ROLE_HIF_EDGE = 2
ROLE_ROOT = 3


@dataclass
class Stage:
    kind: int
    in_len: int
    out_len: int
    role: int = ROLE_BF
    level: int = 0
    blocks: list = field(default_factory=list)  # (M[rows, cols], inp[cols], out[rows])

    def add(self, M, inp, out):
        M = np.asarray(M, dtype=np.complex128)
        inp = np.asarray(inp, dtype=np.int64)
        out = np.asarray(out, dtype=np.int64)
        assert M.shape == (len(out), len(inp)), (M.shape, len(out), len(inp))
        self.blocks.append((M, inp, out))

    @property
    def nnz(self) -> int:
        return sum(M.size for M, _, _ in self.blocks)

    def padded_shape(self):
        R = max((len(o) for _, _, o in self.blocks), default=0)
        C = max((len(i) for _, i, _ in self.blocks), default=0)
        if self.kind == KIND_INPLACE:
            R = C = max(R, C)
        return R, C

    def apply(self, x: np.ndarray, adjoint: bool = False) -> np.ndarray:
        """Reference product used inside the builder (peeling probes); not the product path."""
        x = np.asarray(x)
        if self.kind == KIND_MAP:
            if not adjoint:
                y = np.zeros((self.out_len,) + x.shape[1:], dtype=np.result_type(x, np.complex128))
                for M, i, o in self.blocks:
                    y[o] = M @ x[i]
            else:
                y = np.zeros((self.in_len,) + x.shape[1:], dtype=np.result_type(x, np.complex128))
                for M, i, o in self.blocks:
                    y[i] = M.conj().T @ x[o]
            return y
        y = np.array(x, dtype=np.result_type(x, np.complex128), copy=True)
        for M, i, o in self.blocks:
            y[i] = (M.conj().T if adjoint else M) @ x[i]
        return y

    def validate(self):
        """Output indices unique (MAP/INPLACE), input indices unique (MAP), sets disjoint."""
        outs = np.concatenate([o for _, _, o in self.blocks]) if self.blocks else np.zeros(0, int)
        ins = np.concatenate([i for _, i, _ in self.blocks]) if self.blocks else np.zeros(0, int)
        assert len(np.unique(outs)) == len(outs), "duplicate output index"
        assert len(np.unique(ins)) == len(ins), "duplicate input index"
        assert outs.size == 0 or (outs.min() >= 0 and outs.max() < self.out_len)
        assert ins.size == 0 or (ins.min() >= 0 and ins.max() < self.in_len)
        if self.kind == KIND_INPLACE:
            for _, i, o in self.blocks:
                assert np.array_equal(i, o)
