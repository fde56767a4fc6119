"""Host factor builder checked against the oracle's definition of K (no GPU).

The factors are the product's; what they are compared with is the oracle's dense K, its LU solve
and the oracle's own product of the packed stages (oracle/factor_apply.py), with the paper's
error measures e_a = ||K - K-dot|| / ||K|| and e_s = ||I - G-dot K-dot* K|| (section 6)."""

import numpy as np
import pytest

from oracle import factor_apply as fa
from oracle import fio_oracle as fo
from paper_2105_02995_gb300.builder import build_operator
from paper_2105_02995_gb300.builder.butterfly import build_butterfly, apply_stages

_cache = {}


def built(kind, n, eb, eh, **kw):
    key = (kind, n, eb, eh, tuple(sorted(kw.items())))
    if key not in _cache:
        _cache[key] = build_operator(kind, n, eb, eh, **kw)
    return _cache[key]


def spec(A):
    return np.linalg.norm(A, 2)


@pytest.mark.parametrize("kind,n,L,eps", [("ex1", 256, 4, 1e-6), ("ex1", 1024, 6, 1e-9),
                                          ("ex2a", 256, 4, 1e-7), ("ex2b", 256, 4, 1e-7),
                                          ("ex3", 16, 2, 1e-4), ("ex3", 32, 3, 1e-6)])
def test_butterfly_error(kind, n, L, eps):
    """e_a of the butterfly within a small multiple of its tolerance (section 2, eq. for K-dot)."""
    st, _ = build_butterfly(kind, n, L, eps)
    op = fo.FIO(kind, n)
    K = fo.dense_K(op)
    Kd = apply_stages(st, np.eye(op.N, dtype=complex))
    assert spec(K - Kd) / spec(K) < 5 * eps


@pytest.mark.parametrize("kind,n,eb,eh,bound", [("ex1", 256, 1e-7, 1e-6, 2e-5), ("ex1", 1024, 1e-7, 1e-6, 5e-5),
                                                ("ex1", 256, 1e-4, 1e-3, 2e-2), ("ex3", 32, 1e-5, 1e-3, 2e-2),
                                                ("ex2a", 256, 1e-7, 1e-6, 1e-3), ("ex2b", 256, 1e-7, 1e-6, 1e-2)])
def test_inverse_error_es(kind, n, eb, eh, bound):
    """e_s = ||I - G-dot K-dot* K|| of the packed operator (the paper reports e_s of the order of
    eps to 10 eps at these sizes, Tables for Examples 1 and 3).  With Example 2's amplitude K*K is
    worse conditioned (cond(K) 17 and 112 at N = 1024 for sigma^2 = 0.1 and 0.05, against 3 for
    Example 1) and e_s grows with it, as in the paper's Example 2 tables (e_s up to 3e-3 at
    eps = 1e-4 for sigma^2 = 0.05): bounds 1e-3 and 1e-2."""
    buf, info = built(kind, n, eb, eh)
    P = fa.PackedFactors(buf)
    op = fo.FIO(kind, n)
    K = fo.dense_K(op)
    GK = fa.apply_inv(P, K)
    es = spec(np.eye(op.N) - GK)
    assert es < bound, es


def test_linear_phase_inverse_is_adjoint_over_N():
    """Phi = x.xi: K*K = N I, so the HIF eliminates every DOF at the leaves (empty root) and
    G-dot K-dot* = K*/N to the butterfly's accuracy (closed form)."""
    buf, info = built("linear1d", 256, 1e-10, 1e-8)
    assert info["root"] == 0
    P = fa.PackedFactors(buf)
    op = fo.FIO("linear1d", 256)
    K = fo.dense_K(op)
    G = fa.dense_G(P)
    assert np.max(np.abs(G - np.eye(256) / 256)) < 1e-12
    assert spec(fa.apply_inv(P, np.eye(256)) - K.conj().T / 256) < 1e-8


@pytest.mark.parametrize("kind,n,eb,eh", [("ex1", 256, 1e-7, 1e-6), ("ex3", 32, 1e-5, 1e-3)])
def test_direct_solve_vs_lu(kind, n, eb, eh):
    """f = G-dot K-dot* u against the dense LU solve: within 10 eps at small N (the paper reports
    e_s of the order of eps to 10 eps at these sizes)."""
    buf, _ = built(kind, n, eb, eh)
    P = fa.PackedFactors(buf)
    op = fo.FIO(kind, n)
    rng = np.random.default_rng(11)
    u = rng.standard_normal((op.N, 3)) + 1j * rng.standard_normal((op.N, 3))
    f = fa.apply_inv(P, u)
    assert fo.rel_err(f, fo.solve_lu(op, u)) < 10 * eh


def test_packed_stages_are_bijections():
    """Every butterfly stage maps onto its output space exactly once in both directions."""
    import struct
    buf, _ = built("ex1", 256, 1e-7, 1e-6)
    nbf = struct.unpack_from("<I", buf, 32)[0]
    tab = struct.unpack_from("<Q", buf, 64)[0]
    for s in range(nbf):
        kind, nblk, R, C = struct.unpack_from("<IIII", buf, tab + 64 * s)
        il, ol = struct.unpack_from("<qq", buf, tab + 64 * s + 16)
        oM, oi, oo = struct.unpack_from("<QQQ", buf, tab + 64 * s + 32)
        ii = np.frombuffer(buf, "<i4", nblk * C, oi)
        jj = np.frombuffer(buf, "<i4", nblk * R, oo)
        assert np.array_equal(np.sort(ii[ii >= 0]), np.arange(il))
        assert np.array_equal(np.sort(jj[jj >= 0]), np.arange(ol))


def test_hmatrix_matches_normal_matrix():
    """Peeling (section 3): S-dot against K-dot* K-dot formed densely, relative error ~ eps."""
    from paper_2105_02995_gb300.builder.hmatrix import HGeometry, peel
    st, _ = build_butterfly("ex1", 256, 4, 1e-8)
    Kd = apply_stages(st, np.eye(256, dtype=complex))
    A = Kd.conj().T @ Kd
    H = peel(lambda X: A @ X, HGeometry(1, 256, 3), 1e-6)
    Sd = H.apply(np.eye(256, dtype=complex))
    assert spec(A - Sd) / spec(A) < 5e-6


def test_butterfly_sampled_path_large_N():
    """N = 16384 uses the sampled middle-level construction (blocks too large for a full SVD):
    K-dot against the oracle's K at sampled rows, relative error within a few eps_BF.  (A random
    row sample once made one block's coefficient solve ill-conditioned; full rows catch that.)"""
    from paper_2105_02995_gb300.builder import PaddedStages
    N, eps = 16384, 1e-7
    st, _ = build_butterfly("ex1", N, 10, eps)
    ps = PaddedStages(st)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2))
    rows = np.sort(rng.choice(N, 48, replace=False))
    got = ps.apply(f)[rows]
    want = fo.K_rows(fo.FIO("ex1", N), rows, f)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 5 * eps


def _node_check(A, nI, M, red, skel, schur):
    """Apply R* = blockdiag(M, I) (M on the node's DOFs in (red, skel) order) to the whole HPD A:
    the redundant block must become the identity and decouple from everything else, and the
    skeleton block must be the returned Schur complement."""
    n = A.shape[0]
    order = np.concatenate([red, skel, np.arange(nI, n)])
    Ap = A[np.ix_(order, order)]
    Rs = np.eye(n, dtype=complex)
    Rs[:nI, :nI] = M
    B = Rs @ Ap @ Rs.conj().T
    nr, ns = len(red), len(skel)
    scale = np.linalg.norm(A, 2)
    assert np.linalg.norm(B[:nr, :nr] - np.eye(nr)) < 1e-10
    assert np.linalg.norm(B[:nr, nr:]) < 1e-9 * scale
    assert np.linalg.norm(B[nr:nr + ns, nr:nr + ns] - schur) < 1e-9 * scale


@pytest.mark.parametrize("rescale", [False, True])
def test_node_factor_decouples_redundant_dofs(rescale):
    """One skeletonization step (section 4.1) on an HPD matrix whose node-to-rest coupling has
    exact rank 3 and whose node block is ill-conditioned (cond ~ 1e6): both the plain ID +
    elimination and the Cholesky-rescaled variant make the redundant block the identity and
    decouple it exactly."""
    from paper_2105_02995_gb300.builder.hif import eliminate, interp_decomp, rescaled_skeletonize
    rng = np.random.default_rng(21)
    nI, nB, r = 12, 20, 3
    Q, _ = np.linalg.qr(rng.standard_normal((nI, nI)) + 1j * rng.standard_normal((nI, nI)))
    AII = (Q * np.logspace(0, -6, nI)) @ Q.conj().T * 50 + 1e-3 * np.eye(nI)
    U = rng.standard_normal((nB, r)) + 1j * rng.standard_normal((nB, r))
    Vt = rng.standard_normal((r, nI)) + 1j * rng.standard_normal((r, nI))
    ABI = 1e-3 * U @ Vt
    ABB = 10 * np.eye(nB) + 0.1 * (lambda X: X @ X.conj().T)(rng.standard_normal((nB, nB)))
    A = np.block([[AII, ABI.conj().T], [ABI, ABB]])
    assert np.linalg.eigvalsh(A).min() > 0
    if rescale:
        red, skel, M, schur = rescaled_skeletonize(AII, ABI, 1e-12)
    else:
        skel, red, T = interp_decomp(ABI, 1e-12, nI)
        M, schur = eliminate(AII, red, skel, T)
    assert len(skel) == r and len(red) == nI - r
    _node_check(A, nI, M, red, skel, schur)


def test_rescaled_hif_accuracy():
    """The Cholesky-rescaled HIF (section 4.1) reaches the standard variant's e_s bounds: Example 1,
    Example 2 (sigma^2 = 0.1) and Example 3; and it reproduces G-dot = I/N exactly for the linear
    phase (K*K = N I: every DOF decouples at the leaves)."""
    for kind, n, eb, eh, bound in (("ex1", 256, 1e-7, 1e-6, 2e-5), ("ex2a", 256, 1e-7, 1e-6, 1e-3),
                                   ("ex3", 32, 1e-5, 1e-3, 2e-2)):
        buf, _ = build_operator(kind, n, eb, eh, hif_rescale=True)
        P = fa.PackedFactors(buf)
        op = fo.FIO(kind, n)
        es = spec(np.eye(op.N) - fa.apply_inv(P, fo.dense_K(op)))
        assert es < bound, (kind, es)
    buf, _ = build_operator("linear1d", 64, 1e-10, 1e-10, hif_rescale=True)
    G = fa.dense_G(fa.PackedFactors(buf))
    assert np.max(np.abs(G - np.eye(64) / 64)) < 1e-12


@pytest.mark.parametrize("kind,n,eb,eh", [("ex1", 256, 1e-7, 1e-6), ("ex3", 16, 1e-5, 1e-3)])
def test_G_is_hermitian_positive_definite(kind, n, eb, eh):
    """G-dot = R_L...R_1 A_0^{-1} R_1*...R_L* is Hermitian positive definite for any invertible node
    factors (A_0 is HPD): the factor oracle's G of a real operator must be, so a node factor applied
    untransposed, in the wrong order, or dropped on one side shows up here."""
    buf, _ = build_operator(kind, n, eb, eh)
    G = fa.dense_G(fa.PackedFactors(buf))
    assert np.linalg.norm(G - G.conj().T) < 1e-12 * np.linalg.norm(G)
    assert np.linalg.eigvalsh(0.5 * (G + G.conj().T)).min() > 0


def test_example3_64_errors_against_the_paper_table():
    """Example 3 at 64^2 (N = 4096) with the paper's eps = 1e-3 and eps_BF = 1e-4, against the
    paper's Table for Example 3 (e_a 9.62e-5, e_s 2.13e-3 at 64^2), both estimated as the paper
    does (section 6: randomized power iteration, here oracle.spectral_norm_est, pinned against
    closed forms) on matrix-free products with the oracle's dense K:
      * e_a = ||K - K-dot|| / ||K|| within 2x the paper's value (measured 1.16e-4);
      * e_s = ||I - G-dot K-dot* K|| within 4x the paper's value: the 2D ID threshold read as
        relative to ||A|| as well (reading R18) eliminates fewer DOFs at 16 x 16 cells than the
        paper's code, and e_s lands at 3x the paper's (measured 6.6e-3; dense SVD 6.6e-3);
        and at most 10 eps.
    G-dot is Hermitian (test_G_is_hermitian_positive_definite), so E* = I - K* K-dot G-dot."""
    n, eb, eh = 64, 1e-4, 1e-3
    buf, info = built("ex3", n, eb, eh)
    P = fa.PackedFactors(buf)
    op = fo.FIO("ex3", n)
    K = fo.dense_K(op)
    N = op.N

    def Dop(x, adj):
        return (fa.apply_Kdot_adj(P, x) - K.conj().T @ x) if adj else (fa.apply_Kdot(P, x) - K @ x)

    ea = fo.spectral_norm_est(Dop, N, iters=30) / fo.spectral_norm_est(
        lambda x, adj: K.conj().T @ x if adj else K @ x, N, iters=30)

    def Eop(x, adj):
        if adj:
            return x - K.conj().T @ fa.apply_Kdot(P, fa.apply_G(P, x))
        return x - fa.apply_inv(P, K @ x)

    es = fo.spectral_norm_est(Eop, N, iters=40)
    assert ea < 2 * 9.62e-5, ea
    assert es < 4 * 2.13e-3 and es < 10 * eh, es
