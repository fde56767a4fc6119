"""Pins of the oracle (oracle/fio_oracle.py) against what the paper and the mathematics fix.

Each test names the fact it checks.  None of them compares the oracle with itself: the expected
values come from hand-worked phases (tests/golden/phase_values.txt), numpy.fft (a library DFT),
closed forms, or an independent elimination.
"""

import os

import numpy as np
import pytest

from oracle import fio_oracle as fo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "phase_values.txt")


def _golden_rows():
    out = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, n, row, col, num, den = line.split()
            out.append((kind, int(n), int(row), int(col), int(num), int(den)))
    return out


def test_golden_phases():
    """Hand-worked entries of K for Examples 1 and 3 (section 6): sign, grids, c(x), ordering."""
    rows = _golden_rows()
    assert len(rows) > 40
    for kind, n, r, c, num, den in rows:
        op = fo.FIO(kind, n)
        got = fo.K_block(op, [r], [c])[0, 0]
        want = np.exp(2j * np.pi * num / den)
        assert abs(got - want) < 1e-14, (kind, n, r, c, got, want)


@pytest.mark.parametrize("kind", ["ex1", "ex3"])
def test_unit_modulus(kind):
    """a = 1 in both examples, so |K_ij| = 1 (eq. 1.6)."""
    op = fo.FIO(kind, 16)
    K = fo.dense_K(op)
    assert np.max(np.abs(np.abs(K) - 1.0)) < 1e-14


@pytest.mark.parametrize("N", [8, 64, 256])
def test_linear_phase_is_inverse_dft_1d(N):
    """Phi = x xi (Example 1 with c = 0): K f = (-1)^i N ifft(f) (library DFT)."""
    op = fo.FIO("linear1d", N)
    rng = np.random.default_rng(1)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    want = ((-1.0) ** np.arange(N)) * N * np.fft.ifft(f)
    assert fo.rel_err(fo.apply_K(op, f), want) < 1e-13
    assert fo.rel_err(fo.dense_K(op) @ f, want) < 1e-13


@pytest.mark.parametrize("n", [4, 8, 16])
def test_linear_phase_is_inverse_dft_2d(n):
    """2D Phi = x.xi with index i1 + n i2: K f = (-1)^(k1+k2) n^2 ifft2(f)."""
    op = fo.FIO("linear2d", n)
    rng = np.random.default_rng(2)
    f = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    F = f.reshape(n, n)  # F[j2, j1]
    k2, k1 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    want = (((-1.0) ** (k1 + k2)) * n * n * np.fft.ifft2(F)).reshape(-1)
    assert fo.rel_err(fo.apply_K(op, f), want) < 1e-13


@pytest.mark.parametrize("kind,n", [("linear1d", 32), ("linear2d", 8)])
def test_linear_phase_normal_matrix_is_NI(kind, n):
    """K*K = N I and K^{-1} = K*/N for the linear phase (closed form)."""
    op = fo.FIO(kind, n)
    S = fo.normal_matrix(op)
    assert np.max(np.abs(S - op.N * np.eye(op.N))) < 1e-10
    rng = np.random.default_rng(3)
    u = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
    assert fo.rel_err(fo.solve_lu(op, u), fo.apply_Kadj(op, u) / op.N) < 1e-12


@pytest.mark.parametrize("kind,n", [("ex1", 64), ("ex1", 256), ("ex3", 8), ("ex3", 16)])
def test_normal_matrix_diag_and_hpd(kind, n):
    """S = K*K: diag(S) = N exactly for a = 1, S Hermitian positive definite (section 3.1)."""
    op = fo.FIO(kind, n)
    S = fo.normal_matrix(op)
    assert np.max(np.abs(np.diag(S) - op.N)) < 1e-9
    assert np.max(np.abs(S - S.conj().T)) < 1e-9
    np.linalg.cholesky(S)  # raises unless positive definite
    assert np.linalg.eigvalsh(S).min() > 0


def test_normal_matrix_decay_ex1():
    """|S(xi, eta)| decays away from the diagonal (Proposition in section 3.1), qualitatively:
    the mean modulus of the band |xi - eta| in [16, 32) is well below the diagonal value N."""
    op = fo.FIO("ex1", 256)
    S = np.abs(fo.normal_matrix(op))
    i, j = np.indices(S.shape)
    band = (np.abs(i - j) >= 16) & (np.abs(i - j) < 32)
    assert S[band].mean() < 0.05 * op.N


def test_adjoint_identity():
    """<K f, u> = <f, K* u> for the matrix-free products (definition of the adjoint)."""
    op = fo.FIO("ex1", 128)
    rng = np.random.default_rng(4)
    f = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
    u = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
    lhs = np.vdot(u, fo.apply_K(op, f))
    rhs = np.vdot(fo.apply_Kadj(op, u), f)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_matrix_free_rows_match_dense():
    """Row-sampled matrix-free K f equals the dense product (chunking has no effect)."""
    op = fo.FIO("ex3", 16)
    K = fo.dense_K(op)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((op.N, 3)) + 1j * rng.standard_normal((op.N, 3))
    rows = np.array([0, 5, 77, 255])
    assert fo.rel_err(fo.K_rows(op, rows, f, chunk=3), (K @ f)[rows]) < 1e-14


def test_gauss_jordan_known_cases():
    """Gauss-Jordan on closed-form systems: a permutation and a 2x2 with a known inverse."""
    P = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], dtype=complex)
    b = np.array([1.0, 2.0, 3.0 + 1j])
    assert np.allclose(fo.gauss_jordan_solve(P, b), [3.0 + 1j, 1.0, 2.0])
    A = np.array([[2, 1j], [-1j, 3]], dtype=complex)  # det = 5, inverse = [[3, -i], [i, 2]] / 5
    Ainv = np.array([[3, -1j], [1j, 2]]) / 5
    assert np.allclose(fo.gauss_jordan_solve(A, np.eye(2)), Ainv, atol=1e-15)


@pytest.mark.parametrize("kind,n", [("ex1", 32), ("ex1", 64), ("ex3", 8)])
def test_lu_matches_gauss_jordan(kind, n):
    """Dense LU solve vs the brute-force elimination at N <= 64."""
    op = fo.FIO(kind, n)
    rng = np.random.default_rng(6)
    u = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
    f_lu = fo.solve_lu(op, u)
    f_gj = fo.gauss_jordan_solve(fo.dense_K(op), u)
    assert fo.rel_err(f_lu, f_gj) < 1e-11
    assert fo.rel_err(fo.apply_K(op, f_lu), u) < 1e-11


def test_cgne_matches_lu():
    """CG on the normal equations (section 5) reaches the LU solution and a small true residual."""
    op = fo.FIO("ex1", 256)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
    K = fo.dense_K(op)
    f, it, res = fo.cgne(op, u, tol=1e-13, K=K)
    assert res < 1e-10
    assert it < 200
    assert fo.rel_err(f, fo.solve_lu(op, u, K=K)) < 1e-9


def test_planted_sign_error_is_caught():
    """A conjugated kernel (wrong sign of the phase) fails the golden and the DFT pins."""
    op = fo.FIO("linear1d", 16)
    K = fo.dense_K(op).conj()
    f = np.arange(16) + 1j
    want = ((-1.0) ** np.arange(16)) * 16 * np.fft.ifft(f)
    assert fo.rel_err(K @ f, want) > 0.1


@pytest.mark.parametrize("n,d", [(8, 1), (64, 1), (4, 2), (8, 2)])
def test_dft_definition_vs_library(n, d):
    """F written out from its definition (section 1) agrees with the numpy.fft path, in both
    directions, for several right-hand sides."""
    rng = np.random.default_rng(11)
    N = n ** d
    f = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
    F = fo.F_matrix(n, d)
    assert fo.rel_err(fo.apply_F(n, d, f), F @ f) < 1e-13
    assert fo.rel_err(fo.apply_Finv(n, d, F @ f), f) < 1e-13
    assert fo.rel_err(fo.apply_Finv(n, d, f), np.linalg.solve(F, f)) < 1e-12


@pytest.mark.parametrize("kind,n", [("linear1d", 32), ("linear2d", 8)])
def test_Finv_is_the_linear_phase_K(kind, n):
    """F^{-1} is the FIO with Phi = x.xi and a = 1 (K built from the phase formula)."""
    op = fo.FIO(kind, n)
    rng = np.random.default_rng(12)
    g = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
    assert fo.rel_err(fo.apply_Finv(n, op.d, g), fo.dense_K(op) @ g) < 1e-13


def test_dft_parseval():
    """||F f||^2 = n^-d ||f||^2 (F is n^{-d/2} times a unitary matrix)."""
    rng = np.random.default_rng(13)
    for n, d in ((64, 1), (16, 2)):
        f = rng.standard_normal(n ** d) + 1j * rng.standard_normal(n ** d)
        lhs = np.linalg.norm(fo.apply_F(n, d, f)) ** 2
        assert abs(lhs - np.linalg.norm(f) ** 2 / n ** d) < 1e-12 * lhs


def test_ex2_amplitude_golden():
    """Example 2's amplitude at hand-worked points (tests/golden/ex2_amplitude.txt): periodic
    distance in x, xi scaled by N, the four centres, sigma^2 of the paper's two tables."""
    path = os.path.join(os.path.dirname(__file__), "golden", "ex2_amplitude.txt")
    sigma2 = {"ex2a": 0.1, "ex2b": 0.05}
    n_rows = 0
    with open(path) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            kind, n, r, c, *q = line.split()
            want = sum(np.exp(-(int(v) / 64.0) / sigma2[kind]) for v in q)
            got = fo.amplitude(fo.FIO(kind, int(n)), [int(r)], [int(c)])[0, 0]
            assert abs(got - want) < 1e-14 * want, (kind, r, c, got, want)
            n_rows += 1
    assert n_rows == 6


@pytest.mark.parametrize("kind", ["ex2a", "ex2b"])
def test_ex2_is_ex1_times_amplitude(kind):
    """|K_ij| = a(x_i, xi_j) > 0 and K / |K| is Example 1's K: the amplitude changes the modulus only."""
    op, op1 = fo.FIO(kind, 64), fo.FIO("ex1", 64)
    K, K1 = fo.dense_K(op), fo.dense_K(op1)
    a = fo.amplitude(op, np.arange(64), np.arange(64))
    assert a.min() > 0
    assert np.max(np.abs(np.abs(K) - a)) < 1e-14
    assert np.max(np.abs(K / np.abs(K) - K1)) < 1e-13


def test_ex2_normal_matrix_hpd_and_harder():
    """K*K stays Hermitian positive definite, and the narrower amplitude (sigma^2 = 0.05) is worse
    conditioned than the wider one, which is worse than Example 1 (the effect the paper's Example 2
    tables show through the iteration counts of CG with K* alone)."""
    conds = {}
    for kind in ("ex1", "ex2a", "ex2b"):
        op = fo.FIO(kind, 128)
        S = fo.normal_matrix(op)
        assert np.max(np.abs(S - S.conj().T)) < 1e-9
        ev = np.linalg.eigvalsh(S)
        assert ev.min() > 0
        conds[kind] = ev.max() / ev.min()
    assert conds["ex1"] < conds["ex2a"] < conds["ex2b"], conds


# ---- planted mistakes: each plausible error in the oracle's K must fail one of its pins ----------

def _golden_mismatches(K_block):
    bad = 0
    for kind, n, r, c, num, den in _golden_rows():
        got = K_block(fo.FIO(kind, n), [r], [c])[0, 0]
        bad += abs(got - np.exp(2j * np.pi * num / den)) > 1e-12
    return bad


def test_planted_mistakes_fail_the_golden_phases():
    """Transposed operand, a dropped phase term, a shifted frequency grid and a wrong sign of the
    smooth part each change hand-worked entries of tests/golden/phase_values.txt."""
    assert _golden_mismatches(fo.K_block) == 0

    def transposed(op, rows, cols):
        return fo.K_block(op, cols, rows)

    def dropped_smooth(op, rows, cols):  # Phi = x.xi only
        lin = fo.FIO("linear1d" if op.d == 1 else "linear2d", op.n)
        return fo.K_block(lin, rows, cols)

    def shifted_grid(op, rows, cols):   # xi = j instead of j - n/2
        k, _ = fo.grid(op, np.asarray(cols))
        shift = np.asarray(cols) + (op.n // 2 if op.d == 1 else (op.n // 2) * (1 + op.n))
        return fo.K_block(op, rows, np.mod(shift, op.N))

    def conj_phase(op, rows, cols):
        return np.conj(fo.K_block(op, rows, cols))

    for wrong in (transposed, dropped_smooth, shifted_grid, conj_phase):
        assert _golden_mismatches(wrong) > 0, wrong.__name__


def test_planted_dft_mistakes_fail_the_definition():
    """A wrong sign of the exponent or a missing (-1)^k modulation in F^{-1} disagrees with the dense
    definition of F (tests above pin apply_Finv against it)."""
    n, d = 16, 1
    rng = np.random.default_rng(14)
    g = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    want = np.linalg.solve(fo.F_matrix(n, d), g)
    assert fo.rel_err(fo.apply_Finv(n, d, g), want) < 1e-12
    no_mod = np.fft.ifft(g) * n                 # (-1)^k modulation dropped
    wrong_sign = _mod(n) * np.fft.fft(g)        # exp(-2 pi i k j / n) instead of exp(+...)
    assert fo.rel_err(no_mod, want) > 0.1
    assert fo.rel_err(wrong_sign, want) > 0.1


def _mod(n):
    return np.where(np.arange(n) % 2 == 0, 1.0, -1.0)


def test_planted_amplitude_mistake_fails_the_golden_amplitudes():
    """A non-periodic distance in x (plain x - x_k) changes the hand-worked Example 2 amplitudes."""
    path = os.path.join(os.path.dirname(__file__), "golden", "ex2_amplitude.txt")
    sigma2 = {"ex2a": 0.1, "ex2b": 0.05}
    bad = 0
    with open(path) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            kind, n, r, c, *q = line.split()
            n, r, c = int(n), int(r), int(c)
            want = sum(np.exp(-(int(v) / 64.0) / sigma2[kind]) for v in q)
            x, eta = r / n, (c - n // 2) / n
            plain = sum(np.exp(-((x - xk) ** 2 + (eta - ek) ** 2) / sigma2[kind]) for xk, ek in fo.EX2_CENTRES)
            bad += abs(plain - want) > 1e-12 * want
    assert bad > 0


def test_cgne_matrix_free_equals_dense():
    """The oracle's matrix-free CG (its mode for N too large for a dense K) follows the same
    iterates as the dense mode: same iteration count, same solution to rounding."""
    op = fo.FIO("ex1", 128)
    rng = np.random.default_rng(15)
    u = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
    f_d, it_d, r_d = fo.cgne(op, u, tol=1e-12, K=fo.dense_K(op))
    f_m, it_m, r_m = fo.cgne(op, u, tol=1e-12)
    assert it_d == it_m
    assert fo.rel_err(f_m, f_d) < 1e-11


# ---- spectral_norm_est: the power iteration behind the e_a / e_s estimates (section 6) --------

@pytest.mark.parametrize("kind,n", [("linear1d", 64), ("linear2d", 8)])
def test_spectral_norm_linear_phase_is_sqrt_N(kind, n):
    """Phi = x.xi: K*K = N I (K is N times a unitary DFT up to signs), so ||K||_2 = sqrt(N).  A
    power iteration that returned the eigenvalue of K*K instead of its square root would give N."""
    op = fo.FIO(kind, n)
    est = fo.spectral_norm_est(lambda x, adj: fo.apply_Kadj(op, x) if adj else fo.apply_K(op, x), op.N, iters=5)
    assert abs(est - np.sqrt(op.N)) < 1e-12 * np.sqrt(op.N)


def test_spectral_norm_closed_forms():
    """Closed forms: a diagonal matrix (the largest modulus, with a spectral gap so that the
    iteration converges), a rank-one matrix u v* (||u|| ||v||, reached after one step), and a
    non-normal matrix whose adjoint must be applied as the conjugate transpose (a planted
    adjoint without the conjugation changes the answer)."""
    d = np.array([0.5, -3.0 + 4.0j, 1.0, 2.0j, 0.1])  # |d| max = 5, next 2
    diag = fo.spectral_norm_est(lambda x, adj: (np.conj(d) if adj else d) * x, 5, iters=60)
    assert abs(diag - 5.0) < 1e-12
    rng = np.random.default_rng(3)
    u = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    v = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    A = np.outer(u, v.conj())
    r1 = fo.spectral_norm_est(lambda x, adj: (A.conj().T if adj else A) @ x, 7, iters=3)
    assert abs(r1 - np.linalg.norm(u) * np.linalg.norm(v)) < 1e-12 * r1
    # [[1, 1j], [0, 1]]: ||A||_2 = (1 + sqrt 5) / 2 (golden ratio; A*A = [[1, 1j], [-1j, 2]])
    B = np.array([[1.0, 1j], [0.0, 1.0]])
    gold = (1 + np.sqrt(5)) / 2
    est = fo.spectral_norm_est(lambda x, adj: (B.conj().T if adj else B) @ x, 2, iters=60)
    assert abs(est - gold) < 1e-12
    wrong = fo.spectral_norm_est(lambda x, adj: (B.T if adj else B) @ x, 2, iters=60)
    assert abs(wrong - gold) > 1e-3
