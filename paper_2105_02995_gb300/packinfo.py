"""Facts about a packed factor buffer (layout: include/fio.h) used for measurement.

Counts, per stage, the true block entries (valid rows x valid columns of each block, i.e. without
the padding) and the vector lengths, from which the bench derives the algorithmic bytes and flops
of every stage launch.  Reads the header and index lists only; no arithmetic of the method.
"""

from __future__ import annotations

import struct

import numpy as np

ROLE_NAMES = {0: "bf", 1: "hif_cell", 2: "hif_edge", 3: "root"}


def stage_table(buf: bytes):
    n_bf, n_hif, n_root = struct.unpack_from("<III", buf, 32)
    tab = struct.unpack_from("<Q", buf, 64)[0]
    out = []
    for s in range(n_bf + n_hif + n_root):
        e = tab + 64 * s
        kind, nblk, R, C = struct.unpack_from("<IIII", buf, e)
        il, ol = struct.unpack_from("<qq", buf, e + 16)
        oM, oi, oo = struct.unpack_from("<QQQ", buf, e + 32)
        level, role = struct.unpack_from("<II", buf, e + 56)
        ii = np.frombuffer(buf, "<i4", nblk * C, oi).reshape(nblk, C)
        jj = np.frombuffer(buf, "<i4", nblk * R, oo).reshape(nblk, R)
        rows = (jj >= 0).sum(axis=1)
        cols = (ii >= 0).sum(axis=1)
        out.append(dict(index=s, kind=kind, nblk=nblk, R=R, C=C, in_len=il, out_len=ol,
                        level=level, role=ROLE_NAMES.get(role, str(role)),
                        nnz=int((rows * cols).sum()), padded=int(nblk * R * C),
                        touched=int(rows.sum())))
    return out


def totals(buf: bytes):
    st = stage_table(buf)
    n_bf = struct.unpack_from("<I", buf, 32)[0]
    P_K = sum(s["nnz"] for s in st[:n_bf])
    P_G = sum(s["nnz"] for s in st[n_bf:])
    return dict(P_K=P_K, P_G=P_G, padded_K=sum(s["padded"] for s in st[:n_bf]),
                padded_G=sum(s["padded"] for s in st[n_bf:]), stages=st, n_bf=n_bf)
