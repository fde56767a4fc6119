"""Pins of the oracle's packed-factor apply (oracle/factor_apply.py).

The buffer here is written by hand with ``struct`` following the layout of include/fio.h, and its
product is worked out by hand, so these tests depend neither on the product's packer nor on the
oracle's own arithmetic.
"""

import numpy as np
import pytest

from oracle import factor_apply as fa

from handpack import hand_pack


def _tiny():
    # stage 1 (MAP): y = [[1,2],[3,4]] applied to (x1, x0)
    s1 = (0, [[[1, 2], [3, 4]]], [[1, 0]], [[0, 1]], 2, 2)
    # stage 2 (MAP, one padded column whose entries must be ignored): z0 = i y1, z1 = 2 y0
    s2 = (0, [[[1j, 99, 0], [0, 99, 2]]], [[1, -1, 0]], [[0, 1]], 2, 2)
    # HIF stage (INPLACE on index 1): x1 <- 5 x1 ; root on {0, 1}: [[2,1],[1,3]]
    h1 = (1, [[[5]]], [[1]], [[1]], 2, 2)
    r0 = (1, [[[2, 1], [1, 3]]], [[0, 1]], [[0, 1]], 2, 2)
    return hand_pack(2, [s1, s2], [h1], [r0])


def test_hand_built_products():
    """K-dot = [[4i, 3i], [4, 2]] and G-dot = diag(1,5) [[2,1],[1,3]] diag(1,5), by hand."""
    P = fa.PackedFactors(_tiny())
    Kd = fa.dense_Kdot(P)
    assert np.allclose(Kd, [[4j, 3j], [4, 2]], atol=0)
    u = np.array([1.0 + 2j, -3.0])
    assert np.allclose(fa.apply_Kdot_adj(P, u), np.array([[-4j, 4], [-3j, 2]]) @ u, atol=1e-15)
    G = fa.dense_G(P)
    assert np.allclose(G, [[2, 5], [5, 75]], atol=0)
    assert np.allclose(fa.apply_inv(P, u), np.array([[2, 5], [5, 75]]) @ (np.array([[-4j, 4], [-3j, 2]]) @ u))


def test_checksum_detects_corruption():
    buf = bytearray(_tiny())
    buf[-300] ^= 0x01
    with pytest.raises(ValueError):
        fa.PackedFactors(bytes(buf))


def test_bad_magic():
    buf = bytearray(_tiny())
    buf[0:8] = b"XXXXXXXX"
    with pytest.raises(ValueError):
        fa.PackedFactors(bytes(buf))



def test_plumbing_operator_stays_in_small_integers():
    """The exact-integer operator of tests/handpack.py: on inputs with integer parts in {-1, 0, 1}
    every intermediate vector of K-dot, K-dot*, G-dot and G-dot K-dot* has integer parts of
    modulus <= 256, which every precision of the library represents exactly (bfloat16 has an
    8-bit significand); the GPU plumbing tests rely on this."""
    from handpack import plumbing_operator
    P = fa.PackedFactors(plumbing_operator())
    rng = np.random.default_rng(0)
    x = rng.integers(-1, 2, (P.N, 6)) + 1j * rng.integers(-1, 2, (P.N, 6))
    # stage by stage, in every order the applies use
    seqs = {"K": [(m, False) for m in P.bf], "Kadj": [(m, True) for m in reversed(P.bf)],
            "G": [(m, False) for m in P.hif] + [(m, False) for m in P.root] + [(m, True) for m in reversed(P.hif)]}
    seqs["inv"] = seqs["Kadj"] + seqs["G"]
    for name, seq in seqs.items():
        v = x.astype(complex)
        for m, adj in seq:
            v = (m.conj().T @ v) if adj else (m @ v)
            for part in (v.real, v.imag):
                assert np.all(part == np.round(part)) and np.abs(part).max() <= 256, name
