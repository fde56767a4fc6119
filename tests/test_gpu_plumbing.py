"""Bit-exact index and permutation plumbing on the GPU.

The operator (tests/handpack.py) is written by hand: signed permutations with a few two-term rows,
on ragged blocks padded inside and at the end of their index lists, with garbage in the padding
entries.  On integer inputs in {-1, 0, 1} (+ i times the same) every product stays a small
integer, exact in every precision, so the CUDA path must equal the oracle's FP64 product of the
same buffer exactly, for every apply (K-dot, K-dot*, G-dot and G-dot K-dot*, the last two with
the in-place HIF stages and their copy-back), every precision, right-hand-side counts on both
sides of the few-right-hand-side kernel (b <= 4) and of the tensor-core threshold (b >= 8),
column-major inputs with ld > N, the host-buffer entry and every kernel variant.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import factor_apply as fa  # noqa: E402
from paper_2105_02995_gb300 import binding, build as fbuild  # noqa: E402

from handpack import plumbing_operator, plumbing_operator_large  # noqa: E402

PRECS = [(binding.FIO_P64, torch.complex128), (binding.FIO_PDF, torch.complex128),
         (binding.FIO_P32, torch.complex64), (binding.FIO_PTF32, torch.complex64),
         (binding.FIO_PBF16, torch.complex64), (binding.FIO_PTF32X3, torch.complex64)]
REFS = {"K": fa.apply_Kdot, "Kadj": fa.apply_Kdot_adj, "G": fa.apply_G, "inv": fa.apply_inv}
FNS = {"K": "fio_apply_K", "Kadj": "fio_apply_Kadj", "G": "fio_apply_G", "inv": "fio_apply_inv"}
_op = {}


def get():
    if "op" not in _op:
        fbuild.build()
        buf = plumbing_operator()
        _op["op"] = (binding.Operator(buf), fa.PackedFactors(buf))
    return _op["op"]


def int_inputs(N, b, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(-1, 2, (N, b)) + 1j * rng.integers(-1, 2, (N, b))


def run(op, what, xd, yd, b, ld, prec):
    lib = binding.load()
    dt = binding.FIO_C128 if xd.dtype == torch.complex128 else binding.FIO_C64
    rc = getattr(lib, FNS[what])(op.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), ld, b, dt,
                                 prec, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, (what, prec, b, binding.STATUS.get(rc, rc))
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec,dtype", PRECS)
@pytest.mark.parametrize("b", [1, 2, 3, 4, 5, 8, 16, 37, 72])
def test_exact_products_match_the_oracle(prec, dtype, b):
    op, P = get()
    x = int_inputs(P.N, b, 1000 + b)
    xd = binding.colmajor(torch.from_numpy(x).to("cuda", dtype))
    for what, ref in REFS.items():
        yd = binding.colmajor(torch.full((P.N, b), 5 - 5j, dtype=dtype, device="cuda"))
        run(op, what, xd, yd, b, P.N, prec)
        got = yd.cpu().numpy().astype(np.complex128)
        assert np.array_equal(got, ref(P, x)), (what, prec, b)


@pytest.mark.parametrize("prec,dtype", PRECS)
@pytest.mark.parametrize("b", [3, 9])
def test_leading_dimension_padding_is_untouched(prec, dtype, b):
    """Column-major vectors with ld = N + 13: the results are exact and the 13 rows between the
    columns keep their contents."""
    op, P = get()
    N, ld = P.N, P.N + 13
    x = int_inputs(N, b, 2000 + b)
    big = torch.zeros((b, ld), dtype=dtype, device="cuda")
    big[:, :N] = torch.from_numpy(x.T.copy()).to("cuda", dtype)
    xd = big.t()[:N]
    for what, ref in REFS.items():
        ybig = torch.full((b, ld), 7 + 7j, dtype=dtype, device="cuda")
        yd = ybig.t()[:N]
        run(op, what, xd, yd, b, ld, prec)
        assert np.array_equal(yd.cpu().numpy().astype(np.complex128), ref(P, x)), (what, prec, b)
        assert torch.all(ybig[:, N:] == 7 + 7j), (what, prec, b)


@pytest.mark.parametrize("b", [2, 6, 40])
def test_host_buffer_entry_is_exact(b):
    op, P = get()
    x = int_inputs(P.N, b, 3000 + b)
    for dt in (np.complex128, np.complex64):
        f = op.apply_inv_host(np.asfortranarray(x.astype(dt)))
        assert np.array_equal(f.astype(np.complex128), fa.apply_inv(P, x)), (dt, b)


@pytest.mark.parametrize("b", [40, 72])
@pytest.mark.parametrize("prec,dtype,variants", [
    (binding.FIO_P64, torch.complex128, list(range(1, 8)) + [13, 14, 15, 16]),
    (binding.FIO_PDF, torch.complex128, list(range(1, 8)) + [14, 15, 16]),
    (binding.FIO_P32, torch.complex64, list(range(1, 8)) + list(range(9, 14)) + [17, 18]),
    (binding.FIO_PTF32, torch.complex64, [20, 21, 22, 30, 31, 32, 33]),
    (binding.FIO_PBF16, torch.complex64, [20, 21, 22, 30, 31, 32, 33]),
    (binding.FIO_PTF32X3, torch.complex64, [20, 21, 22, 30, 31, 32, 33])])
def test_every_kernel_variant_is_exact(prec, dtype, variants, b):
    op, P = get()
    x = int_inputs(P.N, b, 4000)
    xd = binding.colmajor(torch.from_numpy(x).to("cuda", dtype))
    want = {w: ref(P, x) for w, ref in REFS.items()}
    try:
        for var in variants:
            op.set_variant(b, prec, var)
            for what in REFS:
                yd = binding.colmajor(torch.empty((P.N, b), dtype=dtype, device="cuda"))
                run(op, what, xd, yd, b, P.N, prec)
                assert np.array_equal(yd.cpu().numpy().astype(np.complex128), want[what]), (var, what)
    finally:
        op.set_variant(b, prec, 0)


def test_few_rhs_kernel_is_exact():
    """Variant 8 (the few-right-hand-side kernel with tree reductions) pinned for b <= 4."""
    op, P = get()
    for prec, dtype in PRECS[:3]:
        for b in (1, 4):
            x = int_inputs(P.N, b, 5000 + b)
            xd = binding.colmajor(torch.from_numpy(x).to("cuda", dtype))
            try:
                op.set_variant(b, prec, 8)
                for what, ref in REFS.items():
                    yd = binding.colmajor(torch.empty((P.N, b), dtype=dtype, device="cuda"))
                    run(op, what, xd, yd, b, P.N, prec)
                    assert np.array_equal(yd.cpu().numpy().astype(np.complex128), ref(P, x)), (prec, b, what)
            finally:
                op.set_variant(b, prec, 0)


_big = {}


@pytest.mark.parametrize("prec", [binding.FIO_PTF32, binding.FIO_PBF16, binding.FIO_PTF32X3, binding.FIO_P32])
@pytest.mark.parametrize("b", [8, 40, 72])
def test_large_exact_operator_every_variant(prec, b):
    """Blocks of 398 x 256 on 64 blocks (many work units per persistent CTA, partial row tiles,
    several right-hand-side tiles): K-dot and K-dot* exact for every kernel variant; a mismatch
    reports the rows and right-hand sides it touches."""
    if "op" not in _big:
        fbuild.build()
        buf = plumbing_operator_large()
        _big["op"] = (binding.Operator(buf), fa.PackedFactors(buf))
    op, P = _big["op"]
    x = int_inputs(P.N, b, 6000 + b)
    xd = binding.colmajor(torch.from_numpy(x).to("cuda", torch.complex64))
    want = {"K": fa.apply_Kdot(P, x), "Kadj": fa.apply_Kdot_adj(P, x)}
    variants = list(range(1, 8)) + list(range(9, 14)) + [17, 18] if prec == binding.FIO_P32 else [0, 20, 30, 31, 32, 33, 40]
    try:
        for var in variants:
            op.set_variant(b, prec, var)
            for what in ("K", "Kadj"):
                yd = binding.colmajor(torch.empty((P.N, b), dtype=torch.complex64, device="cuda"))
                run(op, what, xd, yd, b, P.N, prec)
                got = yd.cpu().numpy().astype(np.complex128)
                bad = np.argwhere(got != want[what])
                assert bad.size == 0, (var, what, len(bad), np.unique(bad[:, 0])[:20], np.unique(bad[:, 1])[:20])
    finally:
        op.set_variant(b, prec, 0)
