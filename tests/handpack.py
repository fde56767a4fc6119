"""Hand-written packed factor buffers for tests (the layout of include/fio.h, written with
``struct`` here, independently of the product's packer).

``hand_pack`` lays out given stage arrays.  ``plumbing_operator`` draws a seeded operator whose
every block is a signed permutation (entries +-1, +-i) with one extra +-1 term in some rows, on
ragged blocks with padding slots inside and at the end of the index lists.  On inputs with
integer parts in {-1, 0, 1} every value along every apply stays an integer of modulus <= 256, so
each precision of the library (FP64, FP32, double-float, TF32, BF16, split TF32) computes it
exactly: the GPU must reproduce the oracle's FP64 product bit for bit, which checks the index
and permutation plumbing (gathers, scatters, padding, layout changes, copy-back of the in-place
stages) independently of rounding.  This module holds no arithmetic of the method.
"""

from __future__ import annotations

import struct

import numpy as np


def checksum(data: bytes) -> int:
    words = struct.unpack("<%dQ" % (len(data) // 8), data)
    return sum(w * (2 * k + 1) for k, w in enumerate(words)) % (1 << 64)


def hand_pack(N, bf, hif, root, d=1, n=None, roles=None):
    """bf/hif/root: lists of (kind, M[nblk,R,C], in[nblk,C], out[nblk,R], in_len, out_len).
    roles: optional role per hif stage (1 cell, 2 edge); butterfly stages get 0, the root 3."""
    stages = bf + hif + root
    role_of = [0] * len(bf) + list(roles or [1] * len(hif)) + [3] * len(root)
    tab = 256
    data = tab + 64 * len(stages)
    data = (data + 255) // 256 * 256
    blobs = []
    entries = []
    cur = data
    for (kind, M, ii, oo, il, ol), role in zip(stages, role_of):
        offs = []
        for arr in (np.asarray(M, "<c16"), np.asarray(ii, "<i4"), np.asarray(oo, "<i4")):
            b = arr.tobytes()
            b += b"\0" * ((-len(b)) % 256)
            offs.append(cur)
            blobs.append(b)
            cur += len(b)
        nblk, R, C = np.asarray(M).shape
        entries.append(struct.pack("<IIIIqqQQQII", kind, nblk, R, C, il, ol, *offs, 0, role))
    body = b"".join(blobs)
    head = bytearray(data)
    head[0:8] = b"FIOPACK1"
    struct.pack_into("<II", head, 8, 1, d)
    struct.pack_into("<qq", head, 16, n if n is not None else N, N)
    struct.pack_into("<IIII", head, 32, len(bf), len(hif), len(root), 0)
    struct.pack_into("<dd", head, 48, 1e-6, 1e-6)
    struct.pack_into("<QQQQ", head, 64, tab, data, data + len(body), checksum(body))
    for s, e in enumerate(entries):
        head[tab + 64 * s: tab + 64 * (s + 1)] = e
    return bytes(head) + body


UNITS = np.array([1, -1, 1j, -1j])


def _slots(rng, valid, total):
    """Positions of `valid` live slots among `total` (the rest padding, -1), padding both inside
    the list and at its end."""
    inner = rng.choice(total - 1, size=valid - 1, replace=False) if valid > 1 else np.array([], int)
    live = np.zeros(total, bool)
    live[np.sort(inner)] = True
    live[total - 2 if total - valid >= 2 else total - 1] = True  # at least one padding slot at the end
    if live.sum() < valid:  # top up deterministically
        for k in range(total):
            if live.sum() == valid:
                break
            live[k] = True
    while live.sum() > valid:
        live[np.flatnonzero(live)[0]] = False
    return live


def _map_stage(rng, in_len, out_len, nblk, R, C, rvalid, cvalid, extra_rows):
    """A MAP stage: nblk blocks, rvalid[k] live rows and cvalid[k] live columns of block k; live
    ins / outs are a permutation of [0, in_len) / [0, out_len).  Every live row takes one live
    column with a unit entry (every live column used at least once when rows >= columns), plus a
    second +-1 term in `extra_rows` rows per block; padding entries hold 7+7j (ignored)."""
    assert sum(rvalid) == out_len and sum(cvalid) == in_len
    pin, pout = rng.permutation(in_len), rng.permutation(out_len)
    M = np.full((nblk, R, C), 7 + 7j)
    ii = -np.ones((nblk, C), int)
    oo = -np.ones((nblk, R), int)
    ci = ro = 0
    for k in range(nblk):
        cl, rl = _slots(rng, cvalid[k], C), _slots(rng, rvalid[k], R)
        ii[k, cl] = pin[ci:ci + cvalid[k]]
        oo[k, rl] = pout[ro:ro + rvalid[k]]
        ci += cvalid[k]
        ro += rvalid[k]
        cols, rows = np.flatnonzero(cl), np.flatnonzero(rl)
        M[k][np.ix_(rows, cols)] = 0
        pick = np.concatenate([rng.permutation(cols), rng.choice(cols, max(0, len(rows) - len(cols)))])
        for r, c in zip(rows, pick[:len(rows)]):
            M[k, r, c] = UNITS[rng.integers(4)]
        for r in rng.choice(rows, min(extra_rows, len(rows)), replace=False):
            free = [c for c in cols if M[k, r, c] == 0]
            if free:
                M[k, r, rng.choice(free)] = rng.choice([1, -1])
    return (0, M, ii, oo, in_len, out_len)


def _inplace_stage(rng, N, sizes, R, extra_rows, pool):
    """An INPLACE stage on disjoint index sets (drawn from `pool`, consumed): block k acts on
    sizes[k] live slots, padded to R."""
    nblk = len(sizes)
    M = np.full((nblk, R, R), 7 + 7j)
    idx = -np.ones((nblk, R), int)
    for k, m in enumerate(sizes):
        live = _slots(rng, m, R)
        take, pool[:] = pool[:m], pool[m:]
        idx[k, live] = take
        pos = np.flatnonzero(live)
        M[k][np.ix_(pos, pos)] = 0
        perm = rng.permutation(pos)
        for r, c in zip(pos, perm):
            M[k, r, c] = UNITS[rng.integers(4)]
        for r in rng.choice(pos, min(extra_rows, len(pos)), replace=False):
            free = [c for c in pos if M[k, r, c] == 0]
            if free:
                M[k, r, rng.choice(free)] = rng.choice([1, -1])
    return (1, M, idx, idx.copy(), N, N)


def plumbing_operator(seed: int = 11, N: int = 96):
    """The seeded exact-integer operator described in the module docstring (1D, N = 96):
    butterfly stages N -> N (6 blocks 20 x 20, 16 live), N -> 128 (8 blocks 16 x 12), 128 -> N
    (4 blocks 24 x 36, 32 live columns); HIF stages on disjoint sets (cells, then edges) and a
    root; every block padded inside and at its end.  Returns the packed bytes."""
    rng = np.random.default_rng(seed)
    s1 = _map_stage(rng, N, N, 6, 20, 20, [16] * 6, [16] * 6, 1)
    s2 = _map_stage(rng, N, 128, 8, 18, 14, [16] * 8, [12] * 8, 1)
    s3 = _map_stage(rng, 128, N, 4, 26, 36, [24] * 4, [32] * 4, 1)
    pool = list(rng.permutation(N))
    h1 = _inplace_stage(rng, N, [10, 12, 9, 11, 8], 14, 1, pool)
    h2 = _inplace_stage(rng, N, [6, 7, 5], 9, 1, pool)
    root = _inplace_stage(rng, N, [18], 20, 1, pool)
    return hand_pack(N, [s1, s2, s3], [h1, h2], [root], roles=[1, 2])


def plumbing_operator_large(seed: int = 12):
    """A butterfly-only exact-integer operator with the block shapes of a 2D middle stage (1D,
    N = 16384): 64 blocks of 398 x 256 live entries (N -> 25472) and back (64 blocks of 256 x 398),
    so that a persistent kernel's CTAs each walk many work units.  Signed permutations with one
    extra +-1 term per block: integer results, exact in every precision."""
    rng = np.random.default_rng(seed)
    N, mid = 16384, 64 * 398
    s1 = _map_stage(rng, N, mid, 64, 400, 258, [398] * 64, [256] * 64, 1)
    s2 = _map_stage(rng, mid, N, 64, 258, 400, [256] * 64, [398] * 64, 1)
    return hand_pack(N, [s1, s2], [], [])
