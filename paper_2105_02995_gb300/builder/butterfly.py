"""Butterfly factorisation K ~ K-dot (section 2), built on the host once per operator.

Structure (section 2, eq. for the nested bases and eq. for K-dot):
  * Middle level: for every X node i at level h and Omega node j at level L-h the block
    K_{ij} ~ U_{ij} D_{ij} V_{ij}^* (rank r_ij, relative tolerance eps).
  * Row side: U_s = U_{s+1} C_s for s = h .. L-1.  For an X node i at level s, a child i_c of i and
    an Omega node j^ at level L-s-1 with children j_k, the block [U_{s;i j_k}(rows of i_c)]_k is
    compressed by a truncated SVD into U_{s+1; i_c j^} C_{s; i_c j^}.
  * Column side: the same recursion on the Omega tree, V_t = V_{t+1} H_t.
  * K-dot = U_L C_{L-1} ... C_h D H*_{L-h} ... H*_{L-1} V_L*.

The middle-level blocks are compressed from sampled columns and rows (entries are evaluated on the
fly; the whole of K is never formed): a random column sample gives an orthonormal range basis Q,
the rows a pivoted QR of Q* selects (plus random rows) give the coefficients by least squares on
Q's sampled rows, and an SVD of the coefficients gives U D V*.  The sample grows until fresh
whole rows and whole columns of the block agree to eps.
This is the build's own construction (the paper uses an external code): any construction with the
structure of the K-dot equation serves, and the result is checked against the dense K.

Each factor becomes one MAP stage (stages.py), L + 3 in all:
  V_L* (leaf points -> coefficients), H*_{L-1} .. H*_{L-h}, D, C_h .. C_{L-1}, U_L (coefficients
  -> leaf points).  Coefficient vectors list the pairs in node-major order with their true ranks.

Weighted variant (the default): the middle singular values are split between both sides
(U sqrt(D), V sqrt(D)) and every nested-basis SVD hands its singular values down with the basis,
so each truncation is relative to what the directions contribute to K rather than to an
orthonormal basis; D is then the identity, a pure permutation of coefficient slots, and is folded
into the index lists of the last H* stage (L + 2 stages).
"""

from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.linalg as sla

from .entries import FIOEntries
from . import blas
from .geometry import Tree
from .stages import KIND_MAP, ROLE_BF, Stage


# range of a sampled block: singular directions above RANGE_REL * eps of the largest are kept (the
# range must be resolved well below eps for the least-squares coefficients to reach eps)
RANGE_REL = 1e-3


def _rank(sv: np.ndarray, eps: float) -> int:
    if sv.size == 0 or sv[0] == 0:
        return 0
    return max(1, int(np.count_nonzero(sv > eps * sv[0])))


def lowrank_block(ent: FIOEntries, P: np.ndarray, Q: np.ndarray, eps: float,
                  rng: np.random.Generator, s0: int = 48, full_limit: int = 1 << 16):
    """K[P, Q] ~ U diag(D) V^* with orthonormal U, V and relative accuracy ~eps."""
    n1, n2 = len(P), len(Q)
    if n1 * n2 <= full_limit:
        U, sv, Vh = np.linalg.svd(ent.block(P, Q), full_matrices=False)
        r = _rank(sv, eps)
        return U[:, :r], sv[:r], Vh[:r].conj().T
    s = s0
    while True:
        sc, sr = min(n2, s), min(n1, s)
        c = np.sort(rng.choice(n2, sc, replace=False))
        Kc = ent.block(P, Q[c])
        Uc, svc, _ = np.linalg.svd(Kc, full_matrices=False)
        k1 = int(np.count_nonzero(svc > RANGE_REL * eps * svc[0]))
        Qb = Uc[:, :k1]
        # rows: the k1 rows a pivoted QR of Qb^* selects (they keep Qb[rho] well conditioned),
        # plus random rows up to the sample size
        piv = sla.qr(Qb.conj().T, mode="r", pivoting=True)[1][:k1]
        extra = rng.choice(np.setdiff1d(np.arange(n1), piv), max(0, sr - k1), replace=False)
        rho = np.sort(np.concatenate([piv, extra]).astype(np.int64))
        Kr = ent.block(P[rho], Q)
        X, *_ = sla.lstsq(Qb[rho], Kr, lapack_driver="gelsy")
        W, sv, Zh = np.linalg.svd(X, full_matrices=False)
        r = _rank(sv, eps)
        U, D, V = Qb @ W[:, :r], sv[:r], Zh[:r].conj().T
        # validation on whole fresh rows and whole fresh columns (an error confined to a few
        # directions shows up in full rows/columns, not necessarily in a small sub-block)
        tr = rng.choice(n1, min(n1, 16), replace=False)
        tc = rng.choice(n2, min(n2, 16), replace=False)
        Tr = ent.block(P[tr], Q)
        Tc = ent.block(P, Q[tc])
        err = max(np.linalg.norm(Tr - (U[tr] * D) @ V.conj().T) / max(np.linalg.norm(Tr), 1e-300),
                  np.linalg.norm(Tc - (U * D) @ V[tc].conj().T) / max(np.linalg.norm(Tc), 1e-300))
        enough = (k1 < sc - 8 or sc == n2) and (k1 < sr - 8 or sr == n1)
        if (enough and err < 10 * eps) or (sc == n2 and sr == n1):
            return U, D, V
        s *= 2


def _workers() -> int:
    return blas.pool_workers()


def _descend(blocks: dict, s0: int, L: int, beta: int, tree: Tree, eps: float, weighted: bool = False):
    """Nested-basis recursion on one side (section 2, eq. U_l = U_{l+1} C_l).

    blocks[(a, b)]: basis (n_a x r) of own-tree node a at level s0 paired with other-tree node b at
    level L - s0.  Returns (transfers, leaves): transfers[s - s0][(a_child, b_parent)] is the
    r' x (sum_k r_{a, b_k}) matrix, leaves[(leaf, 0)] the final leaf bases.
    """
    transfers = []
    with blas.threads(1), ThreadPoolExecutor(_workers()) as ex:
        for s in range(s0, L):
            rows = tree.size(s + 1)

            def one(a, s=s, rows=rows, blocks=blocks):
                res = []
                for bp in range(beta ** (L - s - 1)):
                    bks = [beta * bp + k for k in range(beta)]
                    for c in range(beta):
                        cat = np.hstack([blocks[(a, bk)][c * rows:(c + 1) * rows] for bk in bks])
                        Uq, sv, Wh = np.linalg.svd(cat, full_matrices=False)
                        r = _rank(sv, eps)
                        if weighted:
                            # keep the singular values with the basis handed to the next level, so
                            # every truncation is relative to what the directions contribute
                            res.append(((beta * a + c, bp), Uq[:, :r] * sv[:r], Wh[:r]))
                        else:
                            res.append(((beta * a + c, bp), Uq[:, :r], sv[:r, None] * Wh[:r]))
                return res

            nxt, T = {}, {}
            for res in ex.map(one, range(beta ** s)):
                for key, U, C in res:
                    nxt[key] = U
                    T[key] = C
            transfers.append(T)
            blocks = nxt
    return transfers, blocks


def _offsets(ranks: dict, n_a: int, n_b: int):
    """Slot offsets of pairs (a, b) listed a-major; returns (offset dict, total length)."""
    off, cur = {}, 0
    for a in range(n_a):
        for b in range(n_b):
            off[(a, b)] = cur
            cur += ranks[(a, b)]
    return off, cur


def build_butterfly(kind: str, n: int, L: int, eps: float, seed: int = 20210506, weighted: bool = True):
    """Factor K for the operator (kind, n) with a depth-L tree at tolerance eps.

    Returns (stages, info): stages in application order for K-dot x (first applied first).
    """
    ent = FIOEntries(kind, n)
    d = ent.d
    tree = Tree(d, n, L)
    beta = tree.beta
    h = L // 2  # X middle level; the Omega middle level is L - h
    # sample size of the first try: the largest rank of a few probe blocks plus oversampling
    nX, nO = beta ** h, beta ** (L - h)
    probe = [(0, 0), (nX // 2, nO // 2), (nX - 1, nO // 3), (nX // 3, nO - 1)]
    r0 = max(lowrank_block(ent, tree.points(h, i), tree.points(L - h, j), eps,
                           np.random.Generator(np.random.PCG64([seed, i, j])))[0].shape[1]
             for i, j in probe)
    s_first = int(1.2 * r0) + 24

    def one(i):
        P = tree.points(h, i)
        res = []
        for j in range(beta ** (L - h)):
            rng = np.random.Generator(np.random.PCG64([seed, i, j]))
            res.append((j, lowrank_block(ent, P, tree.points(L - h, j), eps, rng, s0=s_first)))
        return i, res

    Ublk, Vblk, Dblk = {}, {}, {}
    with blas.threads(1), ThreadPoolExecutor(_workers()) as ex:
        for i, res in ex.map(one, range(beta ** h)):
            for j, (U, D, V) in res:
                Ublk[(i, j)] = U
                Vblk[(j, i)] = V
                Dblk[(i, j)] = D

    if weighted:
        # K_ij = (U sqrt D)(V sqrt D)^*: both sides carry the weights, the middle factor is I
        for key in Ublk:
            w = np.sqrt(Dblk[key])
            Ublk[key] = Ublk[key] * w
            Vblk[(key[1], key[0])] = Vblk[(key[1], key[0])] * w
            Dblk[key] = np.ones_like(w)
    Ctr, Uleaf = _descend(Ublk, h, L, beta, tree, eps, weighted)
    Htr, Vleaf = _descend(Vblk, L - h, L, beta, tree, eps, weighted)

    # ranks per level on each side: Ur[s][(i, j)] at X-level s; Vr[t][(j, i)] at Omega-level t
    Ur = {h: {k: v.shape[1] for k, v in Ublk.items()}}
    for s in range(h + 1, L + 1):
        src = Ctr[s - h - 1]
        Ur[s] = {k: v.shape[0] for k, v in src.items()}
    Vr = {L - h: {k: v.shape[1] for k, v in Vblk.items()}}
    for t in range(L - h + 1, L + 1):
        src = Htr[t - (L - h) - 1]
        Vr[t] = {k: v.shape[0] for k, v in src.items()}
    Uoff = {s: _offsets(Ur[s], beta ** s, beta ** (L - s)) for s in Ur}
    Voff = {t: _offsets(Vr[t], beta ** t, beta ** (L - t)) for t in Vr}

    def uslots(s, i, j):
        o = Uoff[s][0][(i, j)]
        return np.arange(o, o + Ur[s][(i, j)])

    def vslots(t, j, i):
        o = Voff[t][0][(j, i)]
        return np.arange(o, o + Vr[t][(j, i)])

    N = tree.N
    stages = []
    # 1. V_L*: Omega leaf points -> coefficients at Omega-level L
    st = Stage(KIND_MAP, N, Voff[L][1], ROLE_BF, level=L)
    for j in range(beta ** L):
        V = Vleaf[(j, 0)]
        st.add(V.conj().T, tree.points(L, j), vslots(L, j, 0))
    stages.append(st)
    # 2. H*_t for t = L-1 .. L-h: Omega-level t+1 coefficients -> Omega-level t.  With weighted
    #    bases the middle factor D is the identity, a permutation of the coefficient slots; it is
    #    folded into the output indices of the last H* stage (which then writes the U slots).
    for t in range(L - 1, L - h - 1, -1):
        Hd = Htr[t - (L - h)]
        fold = weighted and t == L - h
        st = Stage(KIND_MAP, Voff[t + 1][1], Uoff[h][1] if fold else Voff[t][1], ROLE_BF, level=t)
        for j in range(beta ** t):
            for ih in range(beta ** (L - t - 1)):
                kids = [beta * j + k for k in range(beta)]
                M = np.hstack([Hd[(jk, ih)].conj().T for jk in kids])
                inp = np.concatenate([vslots(t + 1, jk, ih) for jk in kids])
                if fold:
                    out = np.concatenate([uslots(h, beta * ih + c, j) for c in range(beta)])
                else:
                    out = np.concatenate([vslots(t, j, beta * ih + c) for c in range(beta)])
                st.add(M, inp, out)
        stages.append(st)
    # 3. D: (j, i) at Omega-level L-h -> (i, j) at X-level h
    if not weighted:
        st = Stage(KIND_MAP, Voff[L - h][1], Uoff[h][1], ROLE_BF, level=h)
        for i in range(beta ** h):
            for j in range(beta ** (L - h)):
                st.add(np.diag(Dblk[(i, j)]), vslots(L - h, j, i), uslots(h, i, j))
        stages.append(st)
    # 4. C_s for s = h .. L-1: X-level s coefficients -> X-level s+1
    for s in range(h, L):
        Cd = Ctr[s - h]
        st = Stage(KIND_MAP, Uoff[s][1], Uoff[s + 1][1], ROLE_BF, level=s)
        for i in range(beta ** s):
            for jh in range(beta ** (L - s - 1)):
                kids = [beta * i + c for c in range(beta)]
                M = np.vstack([Cd[(ic, jh)] for ic in kids])
                inp = np.concatenate([uslots(s, i, beta * jh + k) for k in range(beta)])
                out = np.concatenate([uslots(s + 1, ic, jh) for ic in kids])
                st.add(M, inp, out)
        stages.append(st)
    # 5. U_L: X-level L coefficients -> X leaf points
    st = Stage(KIND_MAP, Uoff[L][1], N, ROLE_BF, level=L)
    for i in range(beta ** L):
        st.add(Uleaf[(i, 0)], uslots(L, i, 0), tree.points(L, i))
    stages.append(st)

    info = {
        "L": L, "h": h, "eps": eps,
        "mid_rank_max": max(v.shape[1] for v in Ublk.values()),
        "mid_rank_mean": float(np.mean([v.shape[1] for v in Ublk.values()])),
        "stage_shapes": [st.padded_shape() for st in stages],
        "nnz": sum(st.nnz for st in stages),
    }
    return stages, info


def apply_stages(stages, x, adjoint=False):
    """Builder-side product of MAP stages (used by the peeling probes on the host)."""
    y = x
    seq = reversed(stages) if adjoint else stages
    for st in seq:
        y = st.apply(y, adjoint)
    return y
