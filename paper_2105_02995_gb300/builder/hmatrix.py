"""Hierarchical-matrix approximation S-dot of K-dot* K-dot by peeling (section 3).

Geometry (section 3.1 and 3.3):
  * 1D: HODLR (weak admissibility): NL(c) = {c}, IL(c) = {sibling of c}.
  * 2D: strong admissibility on the quadtree of Omega, periodic in both directions (the paper adds
    the cells that become adjacent after wrapping the domain to NL): NL(c) = the 3 x 3 periodic
    neighbourhood, IL(c) = children of NL(parent(c)) minus NL(c).

Peeling (section 3.2 for 1D, 3.3 for 2D), levels l = 1 .. L_H:
  * colour classes: 1D cells by parity; 2D the 64 sets P_pq = {cells with a1 = p, a2 = q mod 8}
    (eq. for P_pq; fewer when the level has fewer cells per side);
  * per class a random probe R (complex Gaussian on the class's cells, zero elsewhere), of
    k + c columns, Y = A R - sum_{l' < l} A-hat_{l'} R;
  * for each admissible pair (c, J in IL(c)) the randomized low-rank formula
    A_Jc ~ U_1 (R_J* U_1)^+ (R_J* A_Jc R_c) (U_2* R_c)^+ U_2* with U_1 = orth(A_Jc R_c) and
    U_2 = orth(A_Jc* R_J) (eq. for the level-1 low-rank block), truncated at eps_peel * ||A||;
  * at the leaves the near-field blocks A_Jc, J in NL(c), are probed with identity columns after
    subtracting every low-rank level (the dense diagonal part D).
The number of probe columns per level grows until every sampled range has rank <= columns - 10.

A is reached only through a product callable mv(X) = K-dot* (K-dot X).
"""

from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import blas
from .geometry import Tree


class HGeometry:
    """NL / IL lists, colour classes and (2D) edges on the Omega tree of depth LH."""

    def __init__(self, d: int, n: int, LH: int):
        self.d, self.n, self.LH = d, n, LH
        self.tree = Tree(d, n, LH)
        self.beta = self.tree.beta
        self.NL = {}
        self.IL = {}
        for lvl in range(LH + 1):
            cnt = self.beta ** lvl
            self.NL[lvl] = [self._nl(lvl, c) for c in range(cnt)]
        for lvl in range(LH + 1):
            cnt = self.beta ** lvl
            if lvl == 0:
                self.IL[0] = [np.zeros(0, dtype=np.int64)]
                continue
            il = []
            for c in range(cnt):
                par = c // self.beta
                kids = np.concatenate([self.beta * p + np.arange(self.beta) for p in self.NL[lvl - 1][par]])
                il.append(np.setdiff1d(np.unique(kids), self.NL[lvl][c]))
            self.IL[lvl] = il

    def _nl(self, lvl: int, c: int) -> np.ndarray:
        if self.d == 1:
            return np.array([c], dtype=np.int64)
        m = 2 ** lvl
        a1, a2 = self.tree.cell_coords(lvl, np.array([c]))
        out = []
        for d1 in (-1, 0, 1):
            for d2 in (-1, 0, 1):
                out.append(self.tree.cell_id(lvl, (a1[0] + d1) % m, (a2[0] + d2) % m))
        return np.unique(np.array(out, dtype=np.int64))

    def classes(self, lvl: int, period: int):
        """Cells of `lvl` grouped by coordinates modulo `period` (capped by the cells per side)."""
        cnt = self.beta ** lvl
        cells = np.arange(cnt)
        coords = self.tree.cell_coords(lvl, cells)
        q = min(period, 2 ** lvl)
        key = coords[0] % q
        if self.d == 2:
            key = key + q * (coords[1] % q)
        return [cells[key == v] for v in np.unique(key)]

    def ancestor(self, lvl: int, c: int, up_lvl: int) -> int:
        return c // (self.beta ** (lvl - up_lvl))


class LowRankLevel:
    """Admissible blocks of one level: pairs (c, J) with c < J, A_Jc ~ U1 B U2^*."""

    def __init__(self):
        self.blocks = {}

    def add(self, c, J, U1, B, U2):
        self.blocks[(c, J)] = (U1, B, U2)

    def apply(self, tree: Tree, lvl: int, X: np.ndarray, Y: np.ndarray, live=None):
        """Y += A-hat_lvl X (both orientations of every stored pair).  `live` (optional boolean
        array over the cells of lvl) marks the cells where X may be nonzero; pairs with no live
        cell contribute nothing and are skipped."""
        for (c, J), (U1, B, U2) in self.blocks.items():
            lc = live is None or live[c]
            lJ = live is None or live[J]
            if not (lc or lJ):
                continue
            pc, pJ = tree.points(lvl, c), tree.points(lvl, J)
            if lc:
                Y[pJ] += U1 @ (B @ (U2.conj().T @ X[pc]))
            if lJ:
                Y[pc] += U2 @ (B.conj().T @ (U1.conj().T @ X[pJ]))

    def get(self, tree: Tree, lvl: int, X: int, Y: int, rows_pos: np.ndarray, cols_pos: np.ndarray):
        """Dense A[rows of X, cols of Y] for an admissible pair; *_pos are local positions."""
        if (Y, X) in self.blocks:  # A_XY with Y < X stored as A_{X,Y} ~ U1 B U2^*
            U1, B, U2 = self.blocks[(Y, X)]
            return U1[rows_pos] @ B @ U2[cols_pos].conj().T
        if (X, Y) in self.blocks:  # A_{Y,X} ~ U1 B U2^*  =>  A_XY = U2 B^* U1^*
            U1, B, U2 = self.blocks[(X, Y)]
            return U2[rows_pos] @ B.conj().T @ U1[cols_pos].conj().T
        return np.zeros((len(rows_pos), len(cols_pos)), dtype=np.complex128)  # rank 0


class HMatrix:
    """Result of peeling: low-rank levels 1..LH and the dense near field at the leaves."""

    def __init__(self, geom: HGeometry, lowrank: dict, near: dict, normA: float):
        self.geom = geom
        self.lowrank = lowrank  # level -> LowRankLevel
        self.near = near  # (c, J) at level LH, J in NL(c) -> A[points(c), points(J)]
        self.normA = normA

    def apply(self, X: np.ndarray) -> np.ndarray:
        """S-dot X (used by tests to compare S-dot with K-dot* K-dot)."""
        t = self.geom.tree
        Y = np.zeros_like(X, dtype=np.complex128)
        for lvl, lr in self.lowrank.items():
            lr.apply(t, lvl, X, Y)
        LH = self.geom.LH
        for (c, J), A in self.near.items():
            Y[t.points(LH, c)] += A @ X[t.points(LH, J)]
        return Y

    def ranks(self):
        return {lvl: max((B.shape[0] for _, B, _ in lr.blocks.values()), default=0)
                for lvl, lr in self.lowrank.items()}


def _orth(Y: np.ndarray, tol: float) -> np.ndarray:
    """Orthonormal basis of the range of Y, directions with singular value above tol."""
    U, sv, _ = np.linalg.svd(Y, full_matrices=False)
    return U[:, : int(np.count_nonzero(sv > tol))]


def _gauss(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def estimate_norm(mv, N: int, rng, iters: int = 12) -> float:
    """||A||_2 of the Hermitian positive semidefinite A by power iteration."""
    x = _gauss(rng, (N, 1))
    lam = 0.0
    for _ in range(iters):
        y = mv(x)
        lam = float(np.linalg.norm(y))
        x = y / lam
    return lam


def peel(mv, geom: HGeometry, eps: float, seed: int = 20210506, s0: int = 24,
         s_max: int = 512, ncl_il: int = None, ncl_near: int = None) -> HMatrix:
    """Peeling of A (reached through mv) into an HMatrix at tolerance eps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tree = geom.tree
    N = tree.N
    LH = geom.LH
    d = geom.d
    if ncl_il is None:
        ncl_il = 2 if d == 1 else 8
    if ncl_near is None:
        ncl_near = 1 if d == 1 else 4
    normA = estimate_norm(mv, N, rng)
    abs_tol = eps * normA
    lowrank = {}

    def subtract(X, upto, cls=None, cls_lvl=None):
        """sum_{l' <= upto} A-hat_l' X for a probe X supported on the cells `cls` of cls_lvl."""
        Y = np.zeros(X.shape, dtype=np.complex128)
        for lv in range(1, upto + 1):
            if lv in lowrank:
                live = None
                if cls is not None:
                    live = np.zeros(geom.beta ** lv, dtype=bool)
                    live[np.asarray(cls) // geom.beta ** (cls_lvl - lv)] = True
                lowrank[lv].apply(tree, lv, X, Y, live)
        return Y

    s = s0
    for lvl in range(1, LH + 1):
        il = geom.IL[lvl]
        if all(len(x) == 0 for x in il):
            lowrank[lvl] = LowRankLevel()
            continue
        while True:
            classes = geom.classes(lvl, ncl_il)
            Ysamp = {}  # (J, c) -> A_Jc R_c
            Rc = {}
            for cls in classes:
                R = np.zeros((N, s), dtype=np.complex128)
                for c in cls:
                    G = _gauss(rng, (tree.size(lvl), s))
                    R[tree.points(lvl, c)] = G
                    Rc[c] = G
                Y = mv(R) - subtract(R, lvl - 1, cls, lvl)
                for c in cls:
                    for J in il[c]:
                        Ysamp[(J, c)] = Y[tree.points(lvl, J)]
            lr = LowRankLevel()
            pairs = [(c, J) for c in range(geom.beta ** lvl) for J in il[c] if J > c]

            def one(cJ, s=s, Ysamp=Ysamp, Rc=Rc):
                c, J = cJ
                Y1 = Ysamp[(J, c)]  # A_Jc R_c
                Y2 = Ysamp[(c, J)]  # A_cJ R_J = A_Jc^* R_J
                # directions of A_Jc above ~abs_tol/10 show up in A_Jc R above ~abs_tol/10 sqrt(s)
                U1 = _orth(Y1, 0.1 * abs_tol * np.sqrt(s))
                U2 = _orth(Y2, 0.1 * abs_tol * np.sqrt(s))
                if U1.shape[1] == 0 or U2.shape[1] == 0:
                    return None
                if max(U1.shape[1], U2.shape[1]) > s - 10 and s < s_max:
                    return "saturated"
                core = Rc[J].conj().T @ Y1  # R_J^* A_Jc R_c
                B = np.linalg.pinv(Rc[J].conj().T @ U1, rcond=1e-12) @ core @ \
                    np.linalg.pinv(U2.conj().T @ Rc[c], rcond=1e-12)
                W, sv, Zh = np.linalg.svd(B, full_matrices=False)
                r = int(np.count_nonzero(sv > abs_tol))
                if r == 0:
                    return None
                return (c, J, U1 @ W[:, :r], np.diag(sv[:r]), U2 @ Zh[:r].conj().T)

            with blas.threads(1), ThreadPoolExecutor(blas.pool_workers()) as ex:
                results = list(ex.map(one, pairs))
            saturated = any(isinstance(x, str) for x in results)
            if not saturated:
                for res in results:
                    if res is not None:
                        lr.add(*res)
            if saturated:
                s = min(2 * s, s_max)
                continue
            lowrank[lvl] = lr
            break

    # leaves: near field by identity probes after removing every low-rank level
    near = {}
    m = tree.size(LH)
    for cls in geom.classes(LH, ncl_near):
        R = np.zeros((N, m), dtype=np.complex128)
        for c in cls:
            R[tree.points(LH, c), np.arange(m)] = 1.0
        Y = mv(R) - subtract(R, LH, cls, LH)
        for c in cls:
            for J in geom.NL[LH][c]:
                near[(J, c)] = Y[tree.points(LH, J)]  # A[points J, points c]
    # symmetrise the near field (A is Hermitian)
    for (J, c), A in list(near.items()):
        if J < c:
            S = 0.5 * (A + near[(c, J)].conj().T)
            near[(J, c)] = S
            near[(c, J)] = S.conj().T
        elif J == c:
            near[(J, c)] = 0.5 * (A + A.conj().T)
    return HMatrix(geom, lowrank, near, normA)
