"""Inverse of the hierarchical matrix S-dot by recursive skeletonization / HIF (section 4).

For l = L_H down to the stop level, on the active DOFs S_l:
  * Cell skeletonization (section 4.1; 4.2 for 2D): for each cell with active DOFs I, build
    U-bar = [A_BI; far-field rows] (eq. for U-bar; in 2D the near field A_BI on the neighbour list
    and, for every level l' <= l, the rows B U* of the admissible blocks of the cell's ancestor,
    eq. for the 2D bases), compute an interpolative decomposition U-bar_{I~} ~ U-bar_{I^} T by
    column-pivoted QR truncated at eps (eq. 4.x, the ID), then the zeroing matrix Z_I and
    the elimination matrix E_I (eq. for Z and eq. for E):
        A~_rr = A_rr - T* A_sr - A_sr* T + T* A_ss T,   A~_sr = A_sr - A_ss T,
        A~_rr = L L*,  W = A~_sr A~_rr^{-1},  A_ss <- A_ss - W A~_sr*.
  * Edge skeletonization (2D only, section 4.2): every active DOF is assigned to the nearest edge
    of its cell; each edge's DOFs (from its two cells) are skeletonized the same way with
    U-bar = [A_BI1 A_BI2; far(I1) (+) far(I2)] (eq. for the edge U-bar).
  * Merge: active DOFs of sibling cells are concatenated (the parent's near field is assembled from
    the children's near blocks and the level-l admissible blocks between them).
Finally A_0, the matrix on the remaining active DOFs, is formed densely and inverted.

Every node contributes the dense matrix (Z_I E_I)* on its index set, ordered (I~, I^):
        (Z E)* = [[L^{-1}, -L^{-1} T*], [-W, I + W T*]],
In general the zeroing is the change of basis x_I = V y~ + P^ y^ whose redundant columns
V span the directions the ID declares decoupled from the rest of the matrix: V = P~ - P^ T for
the ID above, and V = C^{-*} (P~ - P^ T') for the Cholesky-rescaled variant of section 4.1
(rescale=True): A_II = C C*, and the ID is taken on the scaled U-bar C^{-*}, so that the block
to eliminate, V* A V = I + T'* T', is well conditioned whatever A_II is (the variant the paper
recommends for ill-conditioned matrices).  The skeleton keeps its columns P^ in both, so the
outside couples to the same DOFs and the rest of the algorithm is unchanged.  Node factor:
        (Z E)* = [[L^{-1} V*], [P^* - W V*]],  V* A V = L L*,  W = (P^* A V) (V* A V)^{-1},
one INPLACE block of the stage R_l* (or Rbar_l*); the root stage holds A_0^{-1}.  Then
        G-dot = R_L ... R_1 A_0^{-1} R_1* ... R_L*   (1D, eq. for G-dot)
and the 2D product with Rbar_l between the cell factors (eq. for G-dot in 2D).
"""

from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.linalg as sla

from . import blas
from .hmatrix import HMatrix
from .stages import KIND_INPLACE, ROLE_HIF_CELL, ROLE_HIF_EDGE, ROLE_ROOT, Stage


def interp_decomp(Ub: np.ndarray, eps: float, ncols: int, abs_tol: float = 0.0):
    """ID by column-pivoted QR: returns (skel positions, redundant positions, T).

    Columns are redundant once the pivoted QR's diagonal falls below max(eps |R_11|, abs_tol)."""
    if Ub.shape[0] == 0 or ncols == 0:
        return np.zeros(0, dtype=np.int64), np.arange(ncols), np.zeros((0, ncols))
    nrm = np.linalg.norm(Ub)
    if nrm == 0:
        return np.zeros(0, dtype=np.int64), np.arange(ncols), np.zeros((0, ncols))
    if Ub.shape[0] > ncols:
        # U-bar = Q R with Q orthonormal: the column ID of R is the column ID of U-bar, and the
        # unpivoted (blocked) QR of a tall matrix is much cheaper than the pivoted one
        Ub = sla.qr(Ub, mode="r", overwrite_a=False, check_finite=False)[0][:ncols]
    Q, R, P = sla.qr(Ub, mode="economic", pivoting=True, check_finite=False)
    diag = np.abs(np.diag(R))
    k = int(np.count_nonzero(diag > max(eps * diag[0], abs_tol))) if diag.size else 0
    if k == 0:
        return np.zeros(0, dtype=np.int64), np.arange(ncols), np.zeros((0, ncols))
    T = sla.solve_triangular(R[:k, :k], R[:k, k:], lower=False)
    return P[:k], P[k:], T


FALLBACKS = [0]


def hpd_factor(A: np.ndarray):
    """(L^{-1}, A^{-1}) for a Hermitian A = L L*.  Cholesky when A is numerically positive
    definite; otherwise (approximation errors can push a tiny eigenvalue below zero) the
    eigendecomposition with eigenvalues floored at 1e-12 max|lambda|, L = Q Lambda^{1/2}.  Any
    square root serves: the node factor (Z E)* is stored densely."""
    try:
        L = np.linalg.cholesky(A)
        Linv = sla.solve_triangular(L, np.eye(L.shape[0], dtype=np.complex128), lower=True)
        return Linv, Linv.conj().T @ Linv
    except np.linalg.LinAlgError:
        FALLBACKS[0] += 1
        lam, Q = np.linalg.eigh(A)
        lam = np.maximum(lam, 1e-12 * np.max(np.abs(lam)))
        Linv = (Q / np.sqrt(lam)).conj().T
        return Linv, (Q / lam) @ Q.conj().T


def eliminate(A: np.ndarray, red: np.ndarray, skel: np.ndarray, T: np.ndarray):
    """Zeroing + Gaussian elimination of the redundant DOFs of one node (eqs. Z, E).

    A: the node's dense block (Hermitian), red/skel: positions.  Returns (M, schur) with M the
    (Z E)* matrix in (red, skel) order and schur the updated A_ss.
    """
    Arr = A[np.ix_(red, red)]
    Asr = A[np.ix_(skel, red)]
    Ass = A[np.ix_(skel, skel)]
    TH = T.conj().T
    Asr_t = Asr - Ass @ T
    Arr_t = Arr - TH @ Asr - Asr.conj().T @ T + TH @ Ass @ T
    Arr_t = 0.5 * (Arr_t + Arr_t.conj().T)
    Linv, Arr_inv = hpd_factor(Arr_t)
    W = Asr_t @ Arr_inv  # A~_sr A~_rr^{-1}
    schur = Ass - W @ Asr_t.conj().T
    schur = 0.5 * (schur + schur.conj().T)
    nr, ns = len(red), len(skel)
    M = np.zeros((nr + ns, nr + ns), dtype=np.complex128)
    M[:nr, :nr] = Linv
    M[:nr, nr:] = -Linv @ TH
    M[nr:, :nr] = -W
    M[nr:, nr:] = np.eye(ns) + W @ TH
    return M, schur


def rescaled_skeletonize(A: np.ndarray, Ub: np.ndarray, eps: float):
    """The Cholesky-rescaled skeletonization of one node (section 4.1): ID of U-bar C^{-*} with
    A = C C*, redundant basis V = C^{-*} (P~ - P^ T'), then the elimination of V* A V.

    Returns (red, skel, M, schur) like interp_decomp + eliminate, or (red, skel, None, None)
    when nothing is redundant."""
    n = A.shape[0]
    Ah = 0.5 * (A + A.conj().T)
    Cinv, _ = hpd_factor(Ah)                     # C^{-1} for A = C C* (any square root)
    CinvH = Cinv.conj().T                        # C^{-*}
    skel, red, T = interp_decomp(Ub @ CinvH, eps, n)
    if len(red) == 0:
        return red, skel, None, None
    nr, ns = len(red), len(skel)
    Y = np.zeros((n, nr), dtype=np.complex128)   # P~ - P^ T'
    Y[red, np.arange(nr)] = 1.0
    Y[skel, :] -= T
    V = CinvH @ Y
    AV = Ah @ V
    Arr_t = V.conj().T @ AV
    Arr_t = 0.5 * (Arr_t + Arr_t.conj().T)
    Asr_t = AV[skel, :]
    Linv, Arr_inv = hpd_factor(Arr_t)
    W = Asr_t @ Arr_inv
    schur = Ah[np.ix_(skel, skel)] - W @ Asr_t.conj().T
    schur = 0.5 * (schur + schur.conj().T)
    order = np.concatenate([red, skel])
    VH = V.conj().T[:, order]                    # V* in (red, skel) column order
    Ps = np.zeros((ns, n), dtype=np.complex128)
    Ps[np.arange(ns), skel] = 1.0
    M = np.empty((n, n), dtype=np.complex128)
    M[:nr] = Linv @ VH
    M[nr:] = Ps[:, order] - W @ VH
    return red, skel, M, schur


class HIF:
    def __init__(self, H: HMatrix, eps: float, edges: bool = None, stop_level: int = None,
                 tol_mode: str = "local", rescale: bool = False):
        self.H = H
        self.g = H.geom
        self.t = self.g.tree
        self.eps = eps
        d = self.g.d
        self.edges = (d == 2) if edges is None else edges
        if stop_level is None:
            stop_level = 1 if d == 1 else 2
        self.stop = min(stop_level, self.g.LH)
        # "local": relative to each node's U-bar (the paper's ID accuracy statement);
        # "global": also accept columns whose residual is below eps ||A||_2
        self.abs_tol = eps * H.normA if tol_mode == "global" else 0.0
        # Cholesky-rescaled skeletonization (section 4.1); its ID is relative to the scaled
        # U-bar, whose block against the node itself is the identity
        self.rescale = rescale
        self.stages = []
        self.stats = []
        self._far_factors()

    # ---- far field -------------------------------------------------------------------------
    def _far_factors(self):
        """Per level l' and cell a: R factor of the stacked B U* rows of a's admissible blocks."""
        self.far = {}
        for lvl, lr in self.H.lowrank.items():
            rows = {}
            for (c, J), (U1, B, U2) in lr.blocks.items():
                rows.setdefault(c, []).append(B @ U2.conj().T)          # A_Jc = U1 (B U2*)
                rows.setdefault(J, []).append(B.conj().T @ U1.conj().T)  # A_cJ = U2 (B* U1*)
            fl = {}
            for a, lst in rows.items():
                F = np.vstack(lst)
                if F.shape[0] > F.shape[1]:
                    F = sla.qr(F, mode="r")[0][: F.shape[1]]
                fl[a] = F
            self.far[lvl] = fl

    def _far_rows(self, lvl: int, c: int, I: np.ndarray) -> list:
        out = []
        pos = self.t.pos[I]
        for up in range(lvl, 0, -1):
            a = self.g.ancestor(lvl, c, up)
            F = self.far.get(up, {}).get(a)
            if F is not None:
                out.append(F[:, pos - a * self.t.size(up)])
        return out

    def _lowrank_block(self, lvl, X, Y, rows, cols):
        """A[rows, cols] for cells X, Y admissible at `lvl` (rows/cols are global DOF ids)."""
        size = self.t.size(lvl)
        return self.H.lowrank[lvl].get(self.t, lvl, X, Y,
                                       self.t.pos[rows] - X * size, self.t.pos[cols] - Y * size)

    # ---- driver ----------------------------------------------------------------------------
    def run(self, verbose: bool = False):
        import time
        g, t = self.g, self.t
        LH = g.LH
        self.dofs = {c: t.points(LH, c).copy() for c in range(g.beta ** LH)}
        self.near = {k: v.copy() for k, v in self.H.near.items()}
        t0 = time.time()
        for lvl in range(LH, self.stop - 1, -1):
            self._cells(lvl)
            if self.edges and lvl >= 2:
                self._edges(lvl)
            if lvl > self.stop:
                self._merge(lvl)
            if verbose:
                print(f"[build]   HIF level {lvl}: {time.time() - t0:.1f} s, active "
                      f"{sum(len(v) for v in self.dofs.values())}", flush=True)
        self._root(self.stop)
        if verbose:
            print(f"[build]   HIF root {self.root_size}: {time.time() - t0:.1f} s, "
                  f"eigen fallbacks {FALLBACKS[0]}", flush=True)
        self.fallbacks = FALLBACKS[0]
        return self.stages

    def _restrict(self, c: int, keep_pos: np.ndarray, lvl: int):
        """Drop eliminated DOFs of cell c from every near block involving c."""
        self.dofs[c] = self.dofs[c][keep_pos]
        for c2 in self.g.NL[lvl][c]:
            if c2 == c:
                self.near[(c, c)] = self.near[(c, c)][np.ix_(keep_pos, keep_pos)]
            else:
                self.near[(c, c2)] = self.near[(c, c2)][keep_pos]
                self.near[(c2, c)] = self.near[(c2, c)][:, keep_pos]

    def _pool(self):
        return ThreadPoolExecutor(blas.pool_workers())

    def _cells(self, lvl: int):
        """Cell skeletonization of every cell of `lvl`.  The cells' index sets are disjoint and each
        elimination changes only its own diagonal block, so all IDs and eliminations are computed
        from the level's starting state (in parallel) and the updates applied afterwards."""
        g = self.g
        st = Stage(KIND_INPLACE, self.t.N, self.t.N, ROLE_HIF_CELL, level=lvl)

        def work(c):
            I = self.dofs[c]
            rows = [self.near[(c2, c)] for c2 in g.NL[lvl][c] if c2 != c]
            rows += self._far_rows(lvl, c, I)
            Ub = np.vstack(rows) if rows else np.zeros((0, len(I)))
            if self.rescale:
                red, skel, M, schur = rescaled_skeletonize(self.near[(c, c)], Ub, self.eps)
                return c, ((red, skel, M, schur) if len(red) else None)
            skel, red, T = interp_decomp(Ub, self.eps, len(I), self.abs_tol)
            if len(red) == 0:
                return c, None
            M, schur = eliminate(self.near[(c, c)], red, skel, T)
            return c, (red, skel, M, schur)

        cells = [c for c in range(g.beta ** lvl) if len(self.dofs[c])]
        with blas.threads(1), self._pool() as ex:
            results = list(ex.map(work, cells))
        nred = 0
        for c, res in results:
            if res is None:
                continue
            red, skel, M, schur = res
            I = self.dofs[c]
            order = np.concatenate([I[red], I[skel]])
            st.add(M, order, order)
            nred += len(red)
            self.near[(c, c)][np.ix_(skel, skel)] = schur
            self._restrict(c, np.sort(skel), lvl)
        if st.blocks:
            self.stages.append(st)
        self.stats.append(("cell", lvl, nred, sum(len(v) for v in self.dofs.values())))

    def _edge_assign(self, lvl: int):
        """Edge of every active DOF: nearest edge of its cell, ties in the order l, r, b, t."""
        n = self.g.n
        m = 2 ** lvl
        s = n // m
        groups = {}
        for c in range(self.g.beta ** lvl):
            I = self.dofs[c]
            if len(I) == 0:
                continue
            a1, a2 = (int(v[0]) for v in self.t.cell_coords(lvl, np.array([c])))
            j1, j2 = I % n, I // n
            dist = np.stack([j1 - a1 * s, (a1 + 1) * s - 1 - j1,
                             j2 - a2 * s, (a2 + 1) * s - 1 - j2], axis=1)
            side = np.argmin(dist, axis=1)
            for sd in range(4):
                sel = np.nonzero(side == sd)[0]
                if len(sel) == 0:
                    continue
                if sd == 0:
                    key = ("v", a1, a2)
                elif sd == 1:
                    key = ("v", (a1 + 1) % m, a2)
                elif sd == 2:
                    key = ("h", a1, a2)
                else:
                    key = ("h", a1, (a2 + 1) % m)
                groups.setdefault(key, {})[c] = I[sel]
        return groups

    def _edge_cells(self, lvl, key):
        t = self.t
        m = 2 ** lvl
        kind, e1, e2 = key
        if kind == "v":
            return int(t.cell_id(lvl, (e1 - 1) % m, e2)), int(t.cell_id(lvl, e1, e2))
        return int(t.cell_id(lvl, e1, (e2 - 1) % m)), int(t.cell_id(lvl, e1, e2))

    def _edges(self, lvl: int):
        """Edge skeletonization (2D): like _cells, every edge is computed from the level's state
        after the cell step, then the Schur complements and removals are applied in order."""
        g, t = self.g, self.t
        st = Stage(KIND_INPLACE, t.N, t.N, ROLE_HIF_EDGE, level=lvl)
        groups = self._edge_assign(lvl)

        def work(key):
            c1, c2 = self._edge_cells(lvl, key)
            p1 = self._pos_of(c1, groups[key].get(c1))
            p2 = self._pos_of(c2, groups[key].get(c2))
            I1, I2 = self.dofs[c1][p1], self.dofs[c2][p2]
            nI1, nI = len(I1), len(I1) + len(I2)
            if nI == 0:
                return None
            cells = np.union1d(g.NL[lvl][c1], g.NL[lvl][c2])
            rows = []
            for cc in cells:
                keep = np.ones(len(self.dofs[cc]), dtype=bool)
                if cc == c1:
                    keep[p1] = False
                if cc == c2:
                    keep[p2] = False
                if not keep.any():
                    continue
                blk = np.zeros((int(keep.sum()), nI), dtype=np.complex128)
                if cc in g.NL[lvl][c1]:
                    blk[:, :nI1] = self.near[(cc, c1)][keep][:, p1]
                if cc in g.NL[lvl][c2]:
                    blk[:, nI1:] = self.near[(cc, c2)][keep][:, p2]
                rows.append(blk)
            for part, (c, I) in enumerate(((c1, I1), (c2, I2))):
                if len(I) == 0:
                    continue
                for F in self._far_rows(lvl, c, I):
                    blk = np.zeros((F.shape[0], nI), dtype=np.complex128)
                    if part == 0:
                        blk[:, :nI1] = F
                    else:
                        blk[:, nI1:] = F
                    rows.append(blk)
            Ub = np.vstack(rows) if rows else np.zeros((0, nI))
            A = np.empty((nI, nI), dtype=np.complex128)
            A[:nI1, :nI1] = self.near[(c1, c1)][np.ix_(p1, p1)]
            A[nI1:, nI1:] = self.near[(c2, c2)][np.ix_(p2, p2)]
            A[:nI1, nI1:] = self.near[(c1, c2)][np.ix_(p1, p2)]
            A[nI1:, :nI1] = self.near[(c2, c1)][np.ix_(p2, p1)]
            if self.rescale:
                red, skel, M, schur = rescaled_skeletonize(A, Ub, self.eps)
                if len(red) == 0:
                    return None
            else:
                skel, red, T = interp_decomp(Ub, self.eps, nI, self.abs_tol)
                if len(red) == 0:
                    return None
                M, schur = eliminate(A, red, skel, T)
            I = np.concatenate([I1, I2])
            return (c1, c2, I, nI1, red, skel, M, schur)

        keys = sorted(groups)
        with blas.threads(1), self._pool() as ex:
            results = list(ex.map(work, keys))
        nred = 0
        for res in results:
            if res is None:
                continue
            c1, c2, I, nI1, red, skel, M, schur = res
            order = np.concatenate([I[red], I[skel]])
            st.add(M, order, order)
            nred += len(red)
            o1 = skel < nI1
            o2 = ~o1
            q1 = self._pos_of(c1, I[skel[o1]])
            q2 = self._pos_of(c2, I[skel[o2]])
            self.near[(c1, c1)][np.ix_(q1, q1)] = schur[np.ix_(o1, o1)]
            self.near[(c2, c2)][np.ix_(q2, q2)] = schur[np.ix_(o2, o2)]
            S12 = schur[np.ix_(o1, o2)]
            self.near[(c1, c2)][np.ix_(q1, q2)] = S12
            self.near[(c2, c1)][np.ix_(q2, q1)] = S12.conj().T
            rr = I[red]
            for c in (c1, c2):
                drop = np.isin(self.dofs[c], rr)
                if drop.any():
                    self._restrict(c, np.nonzero(~drop)[0], lvl)
        if st.blocks:
            self.stages.append(st)
        self.stats.append(("edge", lvl, nred, sum(len(v) for v in self.dofs.values())))

    def _pos_of(self, c, ids):
        """Positions in dofs[c] of the global DOF ids `ids` (all still active)."""
        if ids is None or len(ids) == 0:
            return np.zeros(0, dtype=np.int64)
        order = np.argsort(self.dofs[c])
        pos = order[np.searchsorted(self.dofs[c], ids, sorter=order)]
        assert np.array_equal(self.dofs[c][pos], ids)
        return pos

    def _merge(self, lvl: int):
        """Concatenate the active DOFs of siblings; assemble the parent level's near field."""
        g = self.g
        beta = g.beta
        plvl = lvl - 1
        dofs, near = {}, {}
        for p in range(beta ** plvl):
            kids = beta * p + np.arange(beta)
            dofs[p] = np.concatenate([self.dofs[c] for c in kids])
        for p in range(beta ** plvl):
            kids = beta * p + np.arange(beta)
            for p2 in g.NL[plvl][p]:
                kids2 = beta * p2 + np.arange(beta)
                blocks = []
                for c in kids:
                    row = []
                    for c2 in kids2:
                        if c2 in g.NL[lvl][c]:
                            row.append(self.near[(c, c2)])
                        else:
                            row.append(self._lowrank_block(lvl, c, c2, self.dofs[c], self.dofs[c2]))
                    blocks.append(row)
                near[(p, p2)] = np.block(blocks) if dofs[p].size and dofs[p2].size else \
                    np.zeros((len(dofs[p]), len(dofs[p2])), dtype=np.complex128)
        self.dofs, self.near = dofs, near

    def _root(self, lvl: int):
        g = self.g
        cells = [c for c in range(g.beta ** lvl) if len(self.dofs[c])]
        S0 = np.concatenate([self.dofs[c] for c in cells]) if cells else np.zeros(0, dtype=np.int64)
        rows = []
        for c in cells:
            row = []
            for c2 in cells:
                if c2 in g.NL[lvl][c]:
                    row.append(self.near[(c, c2)])
                else:
                    row.append(self._far_pair(lvl, c, c2))
            rows.append(row)
        st = Stage(KIND_INPLACE, self.t.N, self.t.N, ROLE_ROOT, level=0)
        if cells:
            A0 = np.block(rows)
            A0 = 0.5 * (A0 + A0.conj().T)
            _, A0inv = hpd_factor(A0)
            A0inv = 0.5 * (A0inv + A0inv.conj().T)
            st.add(A0inv, S0, S0)
        self.root_size = len(S0)
        self.stages.append(st)

    def _far_pair(self, lvl, c, c2):
        """A[dofs c, dofs c2] for cells not in each other's NL at `lvl`: find the admissible level."""
        for up in range(lvl, 0, -1):
            a = self.g.ancestor(lvl, c, up)
            a2 = self.g.ancestor(lvl, c2, up)
            if a2 in self.g.IL[up][a]:
                size = self.t.size(up)
                return self.H.lowrank[up].get(self.t, up, a, a2,
                                              self.t.pos[self.dofs[c]] - a * size,
                                              self.t.pos[self.dofs[c2]] - a2 * size)
        raise RuntimeError("cells neither near nor admissible")


def build_hif(H: HMatrix, eps: float, verbose: bool = False, **kw):
    h = HIF(H, eps, **kw)
    return h.run(verbose), h
