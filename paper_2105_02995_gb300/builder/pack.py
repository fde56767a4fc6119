"""Stage-major packing of the factors into one flat little-endian buffer (layout: include/fio.h).

Header (256 bytes), stage table (64 bytes per stage), then per stage three 256-byte-aligned
arrays: the blocks M[nblk][R][C] (complex128, row-major inside a block, zero padded), the input
index lists in[nblk][C] and the output index lists out[nblk][R] (int32, -1 = padding).
Stage order: the butterfly stages of K-dot (first applied first), the HIF stages in the order
R_L*, (Rbar_L*), ..., R_1*, (Rbar_1*), then the root stage A_0^{-1}.
A checksum over the data region lets the loader reject a damaged buffer.
"""

from __future__ import annotations

import struct

import numpy as np

from .stages import KIND_INPLACE, Stage

MAGIC = b"FIOPACK1"
VERSION = 1
HEADER_BYTES = 256
STAGE_BYTES = 64
ALIGN = 256


def checksum(buf, start: int, end: int) -> int:
    """Sum over the little-endian u64 words w_k of [start, end) of w_k * (2k + 1), mod 2^64."""
    words = np.frombuffer(buf, dtype="<u8", count=(end - start) // 8, offset=start)
    k = np.arange(len(words), dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(words * (np.uint64(2) * k + np.uint64(1)), dtype=np.uint64))


def _stage_arrays(st: Stage):
    R, C = st.padded_shape()
    # even padded widths keep every block row 16-byte aligned in the complex64 copy
    R, C = R + (R & 1), C + (C & 1)
    nb = len(st.blocks)
    M = np.zeros((nb, R, C), dtype="<c16")
    ii = np.full((nb, C), -1, dtype="<i4")
    oo = np.full((nb, R), -1, dtype="<i4")
    for b, (blk, inp, out) in enumerate(st.blocks):
        r, c = blk.shape
        M[b, :r, :c] = blk
        ii[b, :c] = inp
        oo[b, :r] = out
        if st.kind == KIND_INPLACE:
            oo[b, :c] = inp
    return M, ii, oo


def pack(d: int, n: int, bf_stages, hif_stages, root_stages, eps_bf: float, eps_hif: float,
         flags: int = 0) -> bytes:
    stages = list(bf_stages) + list(hif_stages) + list(root_stages)
    for st in stages:
        st.validate()
    N = n ** d
    tab = HEADER_BYTES
    data = -(-(tab + STAGE_BYTES * len(stages)) // ALIGN) * ALIGN
    cur = data
    entries, blobs = [], []
    for st in stages:
        M, ii, oo = _stage_arrays(st)
        offs = []
        for arr in (M, ii, oo):
            b = arr.tobytes()
            b += b"\0" * ((-len(b)) % ALIGN)
            offs.append(cur)
            blobs.append(b)
            cur += len(b)
        nb, R, C = M.shape
        entries.append(struct.pack("<IIIIqqQQQII", st.kind, nb, R, C, st.in_len, st.out_len,
                                   offs[0], offs[1], offs[2], st.level, st.role))
    out = bytearray(cur)
    out[0:8] = MAGIC
    struct.pack_into("<II", out, 8, VERSION, d)
    struct.pack_into("<qq", out, 16, n, N)
    struct.pack_into("<IIII", out, 32, len(bf_stages), len(hif_stages), len(root_stages), flags)
    struct.pack_into("<dd", out, 48, eps_bf, eps_hif)
    pos = data
    for b in blobs:
        out[pos:pos + len(b)] = b
        pos += len(b)
    struct.pack_into("<QQQQ", out, 64, tab, data, cur, checksum(out, data, cur))
    for s, e in enumerate(entries):
        out[tab + STAGE_BYTES * s: tab + STAGE_BYTES * (s + 1)] = e
    return bytes(out)
