"""Entry evaluation of the discrete FIO for the factor builder.

K_ij = a(x_i, xi_j) exp(2 pi i Phi(x_i, xi_j)) (section 1, eq. 1.6) with the operators of
section 6: Example 1 (1D, a = 1, Phi = x xi + c(x)|xi|, c = (2 + sin 2 pi x)/8), Example 2 (the
phase of Example 1 with a variable amplitude: a mixture of four Gaussians in (x, xi/N), periodic
in x, centres ((2k+1)/8, (2k-3)/8), width sigma^2 = 0.1 for "ex2a" and 0.05 for "ex2b"; the
paper leaves the number of terms, the centres and the scale of xi open), Example 3 (2D
generalized Radon transform, a = 1, Phi = x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2)), and the linear
phase Phi = x.xi (Example 1 with c = 0).  Grid: x = k/n, xi = k - n/2, linear index i1 + n*i2.

The builder evaluates sampled rows and columns of K, never the whole matrix.  The per-point
quantities (integer coordinates, c(x)) are precomputed once.  The exact part x.xi is reduced in
integers modulo n; the smooth part is reduced by its nearest integer before the exponential.
"""

from __future__ import annotations

import numpy as np

KINDS = {"ex1": 1, "ex2a": 1, "ex2b": 1, "linear1d": 1, "ex3": 2, "linear2d": 2}
_GAUSS_WIDTH2 = {"ex2a": 0.1, "ex2b": 0.05}
_GAUSS_CENTRES = tuple(((2 * k + 1) / 8.0, (2 * k - 3) / 8.0) for k in range(4))


class FIOEntries:
    def __init__(self, kind: str, n: int):
        if kind not in KINDS:
            raise ValueError(f"unknown operator kind {kind!r}")
        self.kind, self.n, self.d = kind, n, KINDS[kind]
        self.N = n ** self.d
        idx = np.arange(self.N, dtype=np.int64)
        if self.d == 1:
            self.k = idx[:, None]
        else:
            self.k = np.stack([idx % n, idx // n], axis=1)
        self.xi = self.k - n // 2
        xs = self.k / n
        self.amp = None
        if kind in ("ex1", "ex2a", "ex2b"):
            self.coef = ((2.0 + np.sin(2 * np.pi * xs[:, 0])) / 8.0)[:, None]
            if kind in _GAUSS_WIDTH2:
                # separable factors of each Gaussian term: g_k(x) (periodic distance), h_k(xi / N)
                w2 = _GAUSS_WIDTH2[kind]
                eta = self.xi[:, 0] / float(self.N)
                gx, hx = [], []
                for xk, ek in _GAUSS_CENTRES:
                    dx = np.mod(xs[:, 0] - xk + 0.5, 1.0) - 0.5
                    gx.append(np.exp(-dx * dx / w2))
                    hx.append(np.exp(-(eta - ek) ** 2 / w2))
                self.amp = (np.stack(gx, axis=1), np.stack(hx, axis=1))
        elif kind == "ex3":
            s1, s2 = np.sin(2 * np.pi * xs[:, 0]), np.sin(2 * np.pi * xs[:, 1])
            c1_, c2_ = np.cos(2 * np.pi * xs[:, 0]), np.cos(2 * np.pi * xs[:, 1])
            self.coef = np.stack([(2.0 + s1 * s2) / 16.0, (2.0 + c1_ * c2_) / 16.0], axis=1)
        else:
            self.coef = None

    def block(self, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
        """K[rows, cols] (rows index X, cols index Omega, natural order)."""
        kr = self.k[rows]
        xc = self.xi[cols]
        lin = kr[:, 0:1] * xc[None, :, 0]
        for t in range(1, self.d):
            lin = lin + kr[:, t:t + 1] * xc[None, :, t]
        lin = np.mod(lin, self.n).astype(np.float64) * (1.0 / self.n)
        if self.kind in ("ex1", "ex2a", "ex2b"):
            sm = self.coef[rows, 0:1] * np.abs(xc[None, :, 0]).astype(np.float64)
        elif self.kind == "ex3":
            a = (self.coef[rows, 0:1] ** 2) * (xc[None, :, 0].astype(np.float64) ** 2)
            b = (self.coef[rows, 1:2] ** 2) * (xc[None, :, 1].astype(np.float64) ** 2)
            sm = np.sqrt(a + b)
        else:
            sm = None
        if sm is not None:
            lin = lin + (sm - np.rint(sm))
        out = np.exp(2j * np.pi * lin)
        if self.amp is not None:
            g, h = self.amp
            out *= g[rows] @ h[cols].T
        return out
