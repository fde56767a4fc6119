"""Oracle apply of a packed factor buffer: the factor products written out as sparse matrices.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the product imports this module,
and this module imports nothing from the product.  It reads the packed buffer byte by byte with
``struct`` (the layout is the one documented in include/fio.h) and never calls the C library.

What it follows:
  * Butterfly factorisation, section 2, eq. (2.x) "K ~ K-dot = U_L C_{L-1} ... C_{L/2} D_{L/2}
    H*_{L/2} ... H*_{L-1} V_L*" and its adjoint "K-dot* = V_L H_{L-1} ... D* C*_{L/2} ... U_L*".
    Each packed butterfly stage is one of these sparse factors (with the tree permutations folded
    into its index lists), so K-dot x is the product of the stage matrices, first stage first,
    and K-dot* x is the product of their conjugate transposes in reverse order.
  * Inverse factorisation, section 4, eq. for G-dot (1D: R_L ... R_1 A_L^{-1} R_1* ... R_L*;
    2D: R_L Rbar_L ... R_1 Rbar_1 A^{-1} Rbar_1* R_1* ... Rbar_L* R_L*).  Each packed HIF stage
    holds, per node, the dense matrix of (Z_I E_I)* on the node's index set I, i.e. one factor
    R_l* (or Rbar_l*) restricted to its nodes; the identity elsewhere (eq. 4.x, the zeroing
    matrix Z and the elimination matrix E).  The root stage holds A_0^{-1} on the remaining
    active DOFs.
  * Direct solver f-hat ~ G-dot K-dot* u (section 5, the inverse factorisation K^{-1} ~ G K*).

Pins (tests/test_factor_apply.py): a hand-built two-stage buffer whose product is worked out by
hand; operators built from the paper's Example 1 / Example 3 whose product is compared with the
dense K of fio_oracle within the paper's error measures e_a = ||K - K-dot||/||K|| and
e_s = ||I - G K-dot* K|| (section 6).
"""

from __future__ import annotations

import struct

import numpy as np
import scipy.sparse as sp

MAGIC = b"FIOPACK1"
HEADER_BYTES = 256
STAGE_BYTES = 64
KIND_MAP = 0
KIND_INPLACE = 1


def _checksum(buf: bytes, start: int, end: int) -> int:
    """Sum over little-endian u64 words w_k of w_k * (2k + 1), modulo 2^64."""
    words = np.frombuffer(buf, dtype="<u8", count=(end - start) // 8, offset=start)
    k = np.arange(len(words), dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(words * (np.uint64(2) * k + np.uint64(1)), dtype=np.uint64))


class PackedFactors:
    """Parsed packed buffer: header fields and, per stage, its sparse matrix."""

    def __init__(self, buf: bytes, verify: bool = True):
        buf = bytes(buf)
        if buf[:8] != MAGIC:
            raise ValueError("bad magic")
        (self.version, self.d) = struct.unpack_from("<II", buf, 8)
        (self.n, self.N) = struct.unpack_from("<qq", buf, 16)
        (self.n_bf, self.n_hif, self.n_root, self.flags) = struct.unpack_from("<IIII", buf, 32)
        (self.eps_bf, self.eps_hif) = struct.unpack_from("<dd", buf, 48)
        (tab, data, total, csum) = struct.unpack_from("<QQQQ", buf, 64)
        if total != len(buf):
            raise ValueError("total_bytes does not match the buffer length")
        if verify and _checksum(buf, data, total) != csum:
            raise ValueError("checksum mismatch")
        self.stages = []
        for s in range(self.n_bf + self.n_hif + self.n_root):
            off = tab + s * STAGE_BYTES
            kind, nblk, R, C = struct.unpack_from("<IIII", buf, off)
            in_len, out_len = struct.unpack_from("<qq", buf, off + 16)
            oM, oi, oo = struct.unpack_from("<QQQ", buf, off + 32)
            M = np.frombuffer(buf, dtype="<c16", count=nblk * R * C, offset=oM).reshape(nblk, R, C)
            ii = np.frombuffer(buf, dtype="<i4", count=nblk * C, offset=oi).reshape(nblk, C)
            oo_ = np.frombuffer(buf, dtype="<i4", count=nblk * R, offset=oo).reshape(nblk, R)
            self.stages.append(self._sparse(kind, M, ii, oo_, in_len, out_len))

    @staticmethod
    def _sparse(kind, M, ii, oo, in_len, out_len):
        """The stage as a scipy sparse matrix of shape (out_len, in_len)."""
        nblk, R, C = M.shape
        rows = np.broadcast_to(oo[:, :, None], (nblk, R, C))
        cols = np.broadcast_to(ii[:, None, :], (nblk, R, C))
        keep = (rows >= 0) & (cols >= 0)
        A = sp.coo_matrix((M[keep], (rows[keep], cols[keep])), shape=(out_len, in_len)).tocsr()
        if kind == KIND_INPLACE:
            # identity on every index that no block of this stage touches
            touched = np.zeros(out_len, dtype=bool)
            touched[oo[oo >= 0]] = True
            eye = sp.diags((~touched).astype(np.complex128), 0, shape=(out_len, in_len))
            A = (A + eye).tocsr()
        return A

    @property
    def bf(self):
        return self.stages[: self.n_bf]

    @property
    def hif(self):
        return self.stages[self.n_bf: self.n_bf + self.n_hif]

    @property
    def root(self):
        return self.stages[self.n_bf + self.n_hif:]


def apply_Kdot(P: PackedFactors, x: np.ndarray) -> np.ndarray:
    """K-dot x: the butterfly stages in order, the first applied to x first."""
    y = np.asarray(x, dtype=np.complex128)
    for S in P.bf:
        y = S @ y
    return y


def apply_Kdot_adj(P: PackedFactors, u: np.ndarray) -> np.ndarray:
    """K-dot* u: conjugate transposes of the butterfly stages, last stage first."""
    y = np.asarray(u, dtype=np.complex128)
    for S in reversed(P.bf):
        y = S.conj().T @ y
    return y


def apply_G(P: PackedFactors, x: np.ndarray) -> np.ndarray:
    """G-dot x = H_1^* ... H_T^* A_0^{-1} H_T ... H_1 x with H_t = the t-th HIF stage (R_l*)."""
    y = np.asarray(x, dtype=np.complex128)
    for S in P.hif:
        y = S @ y
    for S in P.root:
        y = S @ y
    for S in reversed(P.hif):
        y = S.conj().T @ y
    return y


def apply_inv(P: PackedFactors, u: np.ndarray) -> np.ndarray:
    """The direct solver f-hat ~ G-dot K-dot* u (section 5)."""
    return apply_G(P, apply_Kdot_adj(P, u))


def dense_Kdot(P: PackedFactors) -> np.ndarray:
    """K-dot as a dense matrix (small N only)."""
    return apply_Kdot(P, np.eye(P.N, dtype=np.complex128))


def dense_G(P: PackedFactors) -> np.ndarray:
    """G-dot as a dense matrix (small N only)."""
    return apply_G(P, np.eye(P.N, dtype=np.complex128))
