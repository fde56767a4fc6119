"""Oracle for the discrete FIO u = K f-hat: the plain definition, in FP64 on the CPU.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the product imports this module.

What it follows (paper section and equation; the paper numbers equations per section):
  * Grids X and Omega: section 1, the definitions of X and Omega (x = n_k/n in [0,1)^d,
    xi integer in [-n/2, n/2)^d, n even).
  * The matrix K_ij = a(x_i, xi_j) exp(2 pi i Phi(x_i, xi_j)): section 1, eq. (1.3) and the
    sentence after eq. (1.6).  No normalisation: the 1/n^d belongs to the DFT F only.
  * Example 1 (section 6): a = 1, Phi = x xi + c(x)|xi|, c(x) = (2 + sin 2 pi x)/8,
    x_i = i/N, xi_j = j - N/2 (the paper writes the same grid 1-based).
  * Example 3 (section 6): a = 1, Phi = x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2),
    c1 = (2 + sin 2pi x1 sin 2pi x2)/16, c2 = (2 + cos 2pi x1 cos 2pi x2)/16.
  * "linear": Phi = x.xi, a = 1 (Example 1 with c = 0).  Then K is diag((-1)^i) times the
    unnormalised inverse DFT (closed form used as a pin).
  * Example 2 (section 6): the phase of Example 1 with a variable amplitude, a mixture of
    Gaussians sum_k exp(-((x - x_k)^2 + (xi - xi_k)^2) / sigma^2), periodic in x on [0, 1],
    sigma^2 = 0.1 ("ex2a") or 0.05 ("ex2b").  The paper gives neither the number of terms nor
    the centres nor the scale of xi; the reading here: four terms, centres
    (x_k, eta_k) = ((2k+1)/8, (2k-3)/8), k = 0..3, with xi measured as eta = xi/N in [-1/2, 1/2)
    and x - x_k as the periodic distance in [-1/2, 1/2).

Readings where the paper is silent:
  * 2D linear index: point (i1, i2) has index i1 + n*i2, for X and for Omega alike.
  * |xi| and the square root are 0 at xi = 0, so that column of K is exp(2 pi i x.xi) = 1.
  * Argument reduction: x.xi = (sum_d i_d xi_d)/n is reduced exactly in integers modulo n;
    the smooth part is reduced by theta - round(theta) before exp(2 pi i theta).

Functions and their pins (tests/test_oracle.py):
  grid, phase_frac, K_block, dense_K      pinned: DFT closed form (numpy.fft), hand-computed
                                          golden rows (tests/golden/), |K_ij| = 1
  apply_K, apply_Kadj, K_rows             pinned: dense product, DFT closed form, <Kf,u> = <f,K*u>
  solve_lu                                pinned: Gauss-Jordan brute force, K^{-1} = K*/N (linear)
  gauss_jordan_solve                      pinned: identity / permutation / closed-form 2x2 cases
  normal_matrix                           pinned: diag = N exactly, Hermitian positive definite,
                                          = N I for the linear phase
  cgne                                    pinned: agrees with solve_lu; true residual
  spectral_norm_est                       the power iteration of the paper's e_a / e_s estimates
                                          (section 6); pinned: ||K||_2 = sqrt(N) for the linear
                                          phase, diagonal, rank-one and a non-normal 2 x 2 closed
                                          form (a planted adjoint without conjugation fails)
  F_matrix, apply_F, apply_Finv           the DFT f-hat = F f of section 1 (definition written out
                                          densely; numpy.fft as the library DFT for large n)
                                          pinned: dense definition vs numpy.fft, F^{-1} = the
                                          linear-phase K (built from the phase formula), Parseval
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg

KINDS = ("ex1", "ex2a", "ex2b", "ex3", "linear1d", "linear2d")
EX2_SIGMA2 = {"ex2a": 0.1, "ex2b": 0.05}
EX2_CENTRES = [((2 * k + 1) / 8.0, (2 * k - 3) / 8.0) for k in range(4)]


@dataclass(frozen=True)
class FIO:
    """A discrete FIO on an n^d grid (section 1).  kind selects the phase of section 6."""

    kind: str
    n: int

    @property
    def d(self) -> int:
        return 1 if self.kind in ("ex1", "ex2a", "ex2b", "linear1d") else 2

    @property
    def N(self) -> int:
        return self.n ** self.d


def grid(op: FIO, idx: np.ndarray):
    """Integer grid coordinates of linear indices idx (same map for X and Omega).

    Returns (k, xi): k[:, t] in [0, n) gives x_t = k_t / n; xi[:, t] = k_t - n/2 in [-n/2, n/2).
    """
    idx = np.asarray(idx, dtype=np.int64)
    n = op.n
    if op.d == 1:
        k = idx[:, None]
    else:
        k = np.stack([idx % n, idx // n], axis=1)
    return k, k - n // 2


def phase_frac(op: FIO, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Phase Phi(x_rows, xi_cols) reduced to [-1/2, 1/2] (only exp(2 pi i Phi) is needed).

    Returns an array of shape (len(rows), len(cols)).
    """
    n = op.n
    kx, _ = grid(op, rows)
    _, xi = grid(op, cols)
    # exact part x.xi = (sum_t k_t * xi_t) / n, reduced modulo n in integers
    num = np.zeros((len(kx), len(xi)), dtype=np.int64)
    for t in range(op.d):
        num += np.outer(kx[:, t], xi[:, t])
    lin = np.mod(num, n).astype(np.float64) / n
    x = kx.astype(np.float64) / n
    if op.kind in ("ex1", "ex2a", "ex2b"):
        c = (2.0 + np.sin(2.0 * np.pi * x[:, 0])) / 8.0
        smooth = np.outer(c, np.abs(xi[:, 0]).astype(np.float64))
    elif op.kind == "ex3":
        s = np.sin(2.0 * np.pi * x)
        co = np.cos(2.0 * np.pi * x)
        c1 = (2.0 + s[:, 0] * s[:, 1]) / 16.0
        c2 = (2.0 + co[:, 0] * co[:, 1]) / 16.0
        xi1 = xi[:, 0].astype(np.float64)
        xi2 = xi[:, 1].astype(np.float64)
        smooth = np.sqrt(np.outer(c1 * c1, xi1 * xi1) + np.outer(c2 * c2, xi2 * xi2))
    elif op.kind in ("linear1d", "linear2d"):
        smooth = np.zeros_like(lin)
    else:
        raise ValueError(f"unknown kind {op.kind!r}")
    smooth = smooth - np.round(smooth)
    theta = lin + smooth
    return theta - np.round(theta)


def amplitude(op: FIO, rows, cols) -> np.ndarray:
    """a(x_rows, xi_cols): 1 except for Example 2 (the Gaussian mixture of the module docstring)."""
    rows, cols = np.asarray(rows), np.asarray(cols)
    if op.kind not in EX2_SIGMA2:
        return np.ones((len(rows), len(cols)))
    kx, _ = grid(op, rows)
    _, xi = grid(op, cols)
    x = kx[:, 0].astype(np.float64) / op.n
    eta = xi[:, 0].astype(np.float64) / op.N
    s2 = EX2_SIGMA2[op.kind]
    a = np.zeros((len(rows), len(cols)))
    for xk, ek in EX2_CENTRES:
        dx = (x - xk + 0.5) % 1.0 - 0.5          # periodic distance in x
        a += np.outer(np.exp(-dx * dx / s2), np.exp(-(eta - ek) ** 2 / s2))
    return a


def K_block(op: FIO, rows, cols) -> np.ndarray:
    """Entries K[rows, cols] = a exp(2 pi i Phi) (eq. 1.3)."""
    theta = phase_frac(op, np.asarray(rows), np.asarray(cols))
    return amplitude(op, rows, cols) * np.exp(2j * np.pi * theta)


def dense_K(op: FIO) -> np.ndarray:
    """The dense N x N matrix K (eq. 1.6)."""
    idx = np.arange(op.N)
    return K_block(op, idx, idx)


def K_rows(op: FIO, rows, f: np.ndarray, chunk: int = 64) -> np.ndarray:
    """(K f)[rows, :] computed one row chunk at a time, O(N) memory per row (matrix-free)."""
    rows = np.asarray(rows, dtype=np.int64)
    f = np.asarray(f, dtype=np.complex128)
    squeeze = f.ndim == 1
    if squeeze:
        f = f[:, None]
    cols = np.arange(op.N)
    out = np.empty((len(rows), f.shape[1]), dtype=np.complex128)
    for s in range(0, len(rows), chunk):
        blk = K_block(op, rows[s:s + chunk], cols)
        out[s:s + chunk] = blk @ f
    return out[:, 0] if squeeze else out


def apply_K(op: FIO, f: np.ndarray, chunk: int = 64) -> np.ndarray:
    """u = K f (eq. 1.6), matrix-free by row chunks."""
    return K_rows(op, np.arange(op.N), f, chunk)


def apply_Kadj(op: FIO, u: np.ndarray, chunk: int = 64) -> np.ndarray:
    """K* u, K* the conjugate transpose of K (adjoint of eq. 1.6)."""
    u = np.asarray(u, dtype=np.complex128)
    squeeze = u.ndim == 1
    if squeeze:
        u = u[:, None]
    cols = np.arange(op.N)
    out = np.zeros((op.N, u.shape[1]), dtype=np.complex128)
    for s in range(0, op.N, chunk):
        rows = np.arange(s, min(op.N, s + chunk))
        blk = K_block(op, rows, cols)
        out += blk.conj().T @ u[rows]
    return out[:, 0] if squeeze else out


def solve_lu(op: FIO, u: np.ndarray, K: np.ndarray | None = None) -> np.ndarray:
    """f-hat = K^{-1} u by dense LU with partial pivoting (LAPACK getrf/getrs as one step)."""
    if K is None:
        K = dense_K(op)
    lu, piv = scipy.linalg.lu_factor(K)
    return scipy.linalg.lu_solve((lu, piv), np.asarray(u, dtype=np.complex128))


def gauss_jordan_solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Brute-force Gauss-Jordan elimination with partial pivoting, row by row in Python.

    For tiny systems only (N <= 64); an independent check of solve_lu.
    """
    A = np.array(A, dtype=np.complex128)
    B = np.array(B, dtype=np.complex128)
    squeeze = B.ndim == 1
    if squeeze:
        B = B[:, None]
    n = A.shape[0]
    aug = [list(A[i]) + list(B[i]) for i in range(n)]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(aug[r][col]))
        if abs(aug[piv][col]) == 0.0:
            raise np.linalg.LinAlgError("singular matrix")
        aug[col], aug[piv] = aug[piv], aug[col]
        p = aug[col][col]
        aug[col] = [v / p for v in aug[col]]
        for r in range(n):
            if r != col and aug[r][col] != 0:
                fac = aug[r][col]
                aug[r] = [a - fac * b for a, b in zip(aug[r], aug[col])]
    X = np.array([row[n:] for row in aug], dtype=np.complex128)
    return X[:, 0] if squeeze else X


def normal_matrix(op: FIO, K: np.ndarray | None = None) -> np.ndarray:
    """S = K* K (section 3.1, the discrete normal matrix)."""
    if K is None:
        K = dense_K(op)
    return K.conj().T @ K


def cgne(op: FIO, u: np.ndarray, tol: float = 1e-13, maxit: int = 500, K: np.ndarray | None = None):
    """Conjugate gradients on K* K f = K* u (the normal equations, section 5), FP64.

    Matrix-free unless a dense K is passed.  Returns (f, iterations, true relative residual
    ||u - K f|| / ||u||) per column.
    """
    u = np.asarray(u, dtype=np.complex128)
    squeeze = u.ndim == 1
    if squeeze:
        u = u[:, None]
    if K is not None:
        mv = lambda v: K @ v  # noqa: E731
        mva = lambda v: K.conj().T @ v  # noqa: E731
    else:
        mv = lambda v: apply_K(op, v)  # noqa: E731
        mva = lambda v: apply_Kadj(op, v)  # noqa: E731
    b = mva(u)
    f = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.sum(np.abs(r) ** 2, axis=0)
    bnorm = np.sqrt(np.sum(np.abs(b) ** 2, axis=0))
    it = 0
    for it in range(1, maxit + 1):
        q = mva(mv(p))
        alpha = rr / np.real(np.sum(p.conj() * q, axis=0))
        f += alpha * p
        r -= alpha * q
        rr_new = np.sum(np.abs(r) ** 2, axis=0)
        if np.all(np.sqrt(rr_new) <= tol * bnorm):
            rr = rr_new
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    res = mv(f) - u
    relres = np.sqrt(np.sum(np.abs(res) ** 2, axis=0)) / np.sqrt(np.sum(np.abs(u) ** 2, axis=0))
    if squeeze:
        return f[:, 0], it, float(relres[0])
    return f, it, relres


def rel_err(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_F / ||b||_F."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def spectral_norm_est(apply, n: int, iters: int = 30, seed: int = 7) -> float:
    """||A||_2 by power iteration on A* A given apply(x, adjoint) -> A x or A* x.

    The paper estimates e_a and e_s by randomized power iteration (section 6)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = apply(apply(x, False), True)
        lam = np.linalg.norm(y)
        if lam == 0:
            return 0.0
        x = y / lam
    return math.sqrt(lam)


# ---- the DFT F of section 1: f-hat(xi) = n^{-d} sum_x exp(-2 pi i x.xi) f(x) ------------------

def F_matrix(n: int, d: int) -> np.ndarray:
    """Dense F (N x N, N = n^d): F[xi, x] = n^{-d} exp(-2 pi i x.xi), x.xi reduced exactly in
    integers modulo n (same grids and 2D index i1 + n*i2 as K)."""
    N = n ** d
    k = np.arange(N)
    if d == 1:
        xi = k - n // 2
        ip = np.outer(xi, k) % n                       # n * (x . xi) mod n, rows xi, cols x
    else:
        x1, x2 = k % n, k // n
        xi1, xi2 = x1 - n // 2, x2 - n // 2
        ip = (np.outer(xi1, x1) + np.outer(xi2, x2)) % n
    return np.exp(-2j * np.pi * ip / n) / N


def _modulation(n: int, d: int) -> np.ndarray:
    """(-1)^(k_1 + ... + k_d): exp(-+2 pi i x.xi) with xi = j - n/2 splits into this sign times
    the standard DFT kernel exp(-+2 pi i k.j / n)."""
    k = np.arange(n ** d)
    s = k % n if d == 1 else (k % n) + (k // n)
    return np.where(s % 2 == 0, 1.0, -1.0)


def apply_F(n: int, d: int, f: np.ndarray) -> np.ndarray:
    """f-hat = F f for f of shape (N,) or (N, b), by numpy.fft (the library DFT)."""
    f = np.asarray(f, dtype=complex)
    vec = f.ndim == 1
    f2 = f.reshape(f.shape[0], -1) * _modulation(n, d)[:, None]
    if d == 1:
        out = np.fft.fft(f2, axis=0) / n
    else:
        b = f2.shape[1]
        out = (np.fft.fft2(f2.reshape(n, n, b), axes=(0, 1)) / (n * n)).reshape(n * n, b)
    return out[:, 0] if vec else out


def apply_Finv(n: int, d: int, fhat: np.ndarray) -> np.ndarray:
    """f = F^{-1} f-hat: f(x) = sum_xi exp(2 pi i x.xi) f-hat(xi), by numpy.fft."""
    g = np.asarray(fhat, dtype=complex)
    vec = g.ndim == 1
    g2 = g.reshape(g.shape[0], -1)
    N = n ** d
    if d == 1:
        out = np.fft.ifft(g2, axis=0) * N
    else:
        b = g2.shape[1]
        out = (np.fft.ifft2(g2.reshape(n, n, b), axes=(0, 1)) * N).reshape(N, b)
    out = out * _modulation(n, d)[:, None]
    return out[:, 0] if vec else out
