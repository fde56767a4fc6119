"""Pins of the oracle's packed-factor apply (oracle/factor_apply.py).

The buffer here is written by hand with ``struct`` following the layout of include/fio.h, and its
product is worked out by hand, so these tests depend neither on the product's packer nor on the
oracle's own arithmetic.
"""

import struct

import numpy as np
import pytest

from oracle import factor_apply as fa


def _checksum(data: bytes) -> int:
    words = struct.unpack("<%dQ" % (len(data) // 8), data)
    return sum(w * (2 * k + 1) for k, w in enumerate(words)) % (1 << 64)


def hand_pack(N, bf, hif, root, d=1):
    """bf/hif/root: lists of (kind, M[nblk,R,C], in[nblk,C], out[nblk,R], in_len, out_len)."""
    stages = bf + hif + root
    tab = 256
    data = tab + 64 * len(stages)
    data = (data + 255) // 256 * 256
    blobs = []
    entries = []
    cur = data
    for kind, M, ii, oo, il, ol in stages:
        offs = []
        for arr in (np.asarray(M, "<c16"), np.asarray(ii, "<i4"), np.asarray(oo, "<i4")):
            b = arr.tobytes()
            b += b"\0" * ((-len(b)) % 256)
            offs.append(cur)
            blobs.append(b)
            cur += len(b)
        nblk, R, C = np.asarray(M).shape
        entries.append(struct.pack("<IIIIqqQQQQ", kind, nblk, R, C, il, ol, *offs, 0))
    body = b"".join(blobs)
    head = bytearray(data)
    head[0:8] = b"FIOPACK1"
    struct.pack_into("<II", head, 8, 1, d)
    struct.pack_into("<qq", head, 16, N, N)
    struct.pack_into("<IIII", head, 32, len(bf), len(hif), len(root), 0)
    struct.pack_into("<dd", head, 48, 1e-6, 1e-6)
    struct.pack_into("<QQQQ", head, 64, tab, data, data + len(body), _checksum(body))
    for s, e in enumerate(entries):
        head[tab + 64 * s: tab + 64 * (s + 1)] = e
    return bytes(head) + body


def _tiny():
    # stage 1 (MAP): y = [[1,2],[3,4]] applied to (x1, x0)
    s1 = (0, [[[1, 2], [3, 4]]], [[1, 0]], [[0, 1]], 2, 2)
    # stage 2 (MAP, one padded column whose entries must be ignored): z0 = i y1, z1 = 2 y0
    s2 = (0, [[[1j, 99, 0], [0, 99, 2]]], [[1, -1, 0]], [[0, 1]], 2, 2)
    # HIF stage (INPLACE on index 1): x1 <- 5 x1 ; root on {0, 1}: [[2,1],[1,3]]
    h1 = (1, [[[5]]], [[1]], [[1]], 2, 2)
    r0 = (1, [[[2, 1], [1, 3]]], [[0, 1]], [[0, 1]], 2, 2)
    return hand_pack(2, [s1, s2], [h1], [r0])


def test_hand_built_products():
    """K-dot = [[4i, 3i], [4, 2]] and G-dot = diag(1,5) [[2,1],[1,3]] diag(1,5), by hand."""
    P = fa.PackedFactors(_tiny())
    Kd = fa.dense_Kdot(P)
    assert np.allclose(Kd, [[4j, 3j], [4, 2]], atol=0)
    u = np.array([1.0 + 2j, -3.0])
    assert np.allclose(fa.apply_Kdot_adj(P, u), np.array([[-4j, 4], [-3j, 2]]) @ u, atol=1e-15)
    G = fa.dense_G(P)
    assert np.allclose(G, [[2, 5], [5, 75]], atol=0)
    assert np.allclose(fa.apply_inv(P, u), np.array([[2, 5], [5, 75]]) @ (np.array([[-4j, 4], [-3j, 2]]) @ u))


def test_checksum_detects_corruption():
    buf = bytearray(_tiny())
    buf[-300] ^= 0x01
    with pytest.raises(ValueError):
        fa.PackedFactors(bytes(buf))


def test_bad_magic():
    buf = bytearray(_tiny())
    buf[0:8] = b"XXXXXXXX"
    with pytest.raises(ValueError):
        fa.PackedFactors(bytes(buf))

