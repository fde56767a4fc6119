"""Host factor builder (Algorithm 1 of the paper): butterfly -> peeling -> HIF -> packed buffer.

``build_operator`` runs once per operator.  It is not on the timed path; its peeling probes can
use the GPU apply of the butterfly through ``mv`` (see binding.Operator.normal_matvec).
"""

from __future__ import annotations

import math
import time

import numpy as np

from .butterfly import build_butterfly
from .hif import build_hif
from .hmatrix import HGeometry, peel
from .pack import pack
from .stages import KIND_MAP

DIMS = {"ex1": 1, "ex2a": 1, "ex2b": 1, "linear1d": 1, "ex3": 2, "linear2d": 2}


class PaddedStages:
    """Batched numpy product of MAP stages from padded block arrays (builder-internal)."""

    def __init__(self, stages):
        self.st = []
        for st in stages:
            assert st.kind == KIND_MAP
            R, C = st.padded_shape()
            nb = len(st.blocks)
            M = np.zeros((nb, R, C), dtype=np.complex128)
            ii = np.full((nb, C), st.in_len, dtype=np.int64)
            oo = np.full((nb, R), st.out_len, dtype=np.int64)
            for b, (blk, i, o) in enumerate(st.blocks):
                M[b, :blk.shape[0], :blk.shape[1]] = blk
                ii[b, :len(i)] = i
                oo[b, :len(o)] = o
            self.st.append((M, ii, oo, st.in_len, st.out_len))

    def apply(self, X: np.ndarray, adjoint: bool = False) -> np.ndarray:
        Y = np.asarray(X, dtype=np.complex128)
        seq = reversed(self.st) if adjoint else self.st
        for M, ii, oo, il, ol in seq:
            src, dst, nin, nout = (oo, ii, ol, il) if adjoint else (ii, oo, il, ol)
            Xp = np.concatenate([Y, np.zeros((1,) + Y.shape[1:], dtype=Y.dtype)])
            G = Xp[src]  # nb x C x s
            Z = np.matmul(M.conj().transpose(0, 2, 1), G) if adjoint else np.matmul(M, G)
            out = np.zeros((nout + 1,) + Y.shape[1:], dtype=np.complex128)
            out[dst] = Z
            Y = out[:nout]
        return Y


def default_levels(kind: str, n: int):
    """Butterfly depth L (leaf 16 points in 1D, 4x4 in 2D) and HIF depth L_H (leaf 64 points in 1D,
    16x16 in 2D, at least one level)."""
    d = DIMS[kind]
    lg = int(round(math.log2(n)))
    if d == 1:
        L = max(2, lg - 4)
        LH = max(1, lg - 6)
    else:
        L = max(2, lg - 2)
        LH = max(1, lg - 4)
    return L, LH


def build_operator(kind: str, n: int, eps_bf: float, eps_hif: float, L: int = None,
                   LH: int = None, mv=None, seed: int = 20210506, verbose: bool = False,
                   hif_rescale: bool = False):
    """Algorithm 1: K-dot <- BFF(eps_bf); S-dot <- peeling(K-dot, eps_hif); G-dot <- HIF(S-dot, eps_hif).

    mv(X) may supply K-dot* K-dot X (e.g. on the GPU); by default the builder's own numpy product
    of the butterfly stages is used.  hif_rescale selects the Cholesky-rescaled skeletonization
    (section 4.1) for the HIF.  Returns (packed bytes, info dict).
    """
    d = DIMS[kind]
    L0, LH0 = default_levels(kind, n)
    L = L0 if L is None else L
    LH = LH0 if LH is None else LH
    t0 = time.time()
    bf, bfinfo = build_butterfly(kind, n, L, eps_bf, seed=seed)
    t1 = time.time()
    if verbose:
        print(f"[build] butterfly {kind} n={n} L={L}: {t1 - t0:.1f} s, max middle rank "
              f"{bfinfo['mid_rank_max']}, {bfinfo['nnz'] / n ** d:.0f} entries per DOF", flush=True)
    if mv is None:
        ps = PaddedStages(bf)
        mv = lambda X: ps.apply(ps.apply(X), adjoint=True)  # noqa: E731
    elif callable(getattr(mv, "bind", None)):
        mv = mv.bind(bf, d, n)
    geom = HGeometry(d, n, LH)
    H = peel(mv, geom, eps_hif, seed=seed + 1)
    t2 = time.time()
    if verbose:
        print(f"[build] peeling L_H={LH}: {t2 - t1:.1f} s, ranks {H.ranks()}", flush=True)
    # 2D: K*K decays only slowly away from the diagonal, so an ID accuracy relative to each node's
    # own U-bar removes few DOFs; accept columns below eps ||A|| as well (the error that matters
    # for the inverse).  1D keeps the node-relative criterion.
    hif_stages, hif = build_hif(H, eps_hif, verbose=verbose,
                                tol_mode="global" if d == 2 else "local", rescale=hif_rescale)
    t3 = time.time()
    if verbose:
        print(f"[build] HIF: {t3 - t2:.1f} s, root {hif.root_size}, steps {hif.stats}", flush=True)
    buf = pack(d, n, bf, hif_stages[:-1], hif_stages[-1:], eps_bf, eps_hif, flags=(d == 2))
    info = dict(kind=kind, n=n, d=d, N=n ** d, L=L, LH=LH, eps_bf=eps_bf, eps_hif=eps_hif,
                hif_rescale=hif_rescale,
                t_bf=t1 - t0, t_peel=t2 - t1, t_hif=t3 - t2, root=hif.root_size,
                nnz_bf=sum(s.nnz for s in bf), nnz_hif=sum(s.nnz for s in hif_stages),
                bf_shapes=[s.padded_shape() for s in bf],
                hif_stats=hif.stats, hmatrix_ranks=H.ranks(), mid_rank_max=bfinfo["mid_rank_max"],
                nbytes=len(buf))
    if verbose:
        print({k: v for k, v in info.items() if k not in ("bf_shapes", "hif_stats")})
    return buf, info


def build_butterfly_only(kind: str, n: int, eps_bf: float, L: int = None, seed: int = 20210506):
    """Packed buffer holding only K-dot (no HIF stages): enough for fio_apply_K / fio_apply_Kadj."""
    d = DIMS[kind]
    L0, _ = default_levels(kind, n)
    bf, info = build_butterfly(kind, n, L0 if L is None else L, eps_bf, seed=seed)
    return pack(d, n, bf, [], [], eps_bf, 0.0, flags=(d == 2)), bf
