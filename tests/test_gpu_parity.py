"""GPU parity: the CUDA path through the C ABI against the oracle, element by element.

Two references, both from oracle/:
  * factor_apply: the same packed factors multiplied out as sparse matrices in FP64.  The FP64
    GPU path must agree to 1e-12 relative; the FP32 path to TOL32 below.  "Relative" is the
    larger of the Frobenius ratio ||a - b|| / ||b|| and the element-wise max|a - b| / max|b|, so
    a few wrong rows cannot hide in the norm of a large array.
  * fio_oracle: the dense K and its LU solve (the plain definition); the direct solve must be
    within 10 eps of it at these sizes, iterative solves must reach the residual they report.
Sizes span several blocks per stage and ragged right-hand-side tiles (b = 1, 3, 5, 16, 37).
Example 3 at n = 64 (N = 4096) is the smallest 2D operator with HIF edge stages (section 4.2,
the edge skeletonization R-bar_l, here at level 2).

TOL32: every stage rounds its outputs to FP32 (unit roundoff 2^-24 ~ 6e-8) after sums of up to
C_max ~ 300 terms, over up to ~20 stages in a row: 20 * sqrt(300) * 6e-8 ~ 2e-5 relative.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import factor_apply as fa  # noqa: E402
from oracle import fio_oracle as fo  # noqa: E402
from paper_2105_02995_gb300 import binding, build as fbuild  # noqa: E402
from paper_2105_02995_gb300.builder import build_operator  # noqa: E402
from paper_2105_02995_gb300.inputs import complex_gaussian, rhs_seed  # noqa: E402

TOL64 = 1e-12
TOL32 = 2e-5

CASES = {
    "ex1_256": ("ex1", 256, 1e-7, 1e-6),     # the 1D N = 256, eps = 1e-6 workload
    "ex1_1024": ("ex1", 1024, 1e-10, 1e-9),
    "ex3_32": ("ex3", 32, 1e-5, 1e-3),
    "ex3_64": ("ex3", 64, 1e-5, 1e-3),       # first size with 2D edge stages
    "ex2b_1024": ("ex2b", 1024, 1e-7, 1e-6),   # Example 2, sigma^2 = 0.05 (variable amplitude)
    "ex3_32_rescaled": ("ex3", 32, 1e-5, 1e-3, True),  # Cholesky-rescaled HIF node factors
}
_ops = {}


def get(name):
    if name not in _ops:
        fbuild.build()
        kind, n, eb, eh, *rescale = CASES[name]
        buf, info = build_operator(kind, n, eb, eh, hif_rescale=bool(rescale and rescale[0]))
        _ops[name] = (buf, info, fa.PackedFactors(buf), binding.Operator(buf), fo.FIO(kind, n))
    return _ops[name]


def dev(a, dtype=torch.complex128):
    return binding.colmajor(torch.from_numpy(np.asarray(a)).to("cuda", dtype))


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def frob(a, b):
    """||a - b||_F / ||b||_F (the norm of the paper's error measures)."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def rel(a, b):
    """max(||a - b||_F / ||b||_F, max|a - b| / max|b|)."""
    a, b = np.asarray(a), np.asarray(b)
    return max(float(np.linalg.norm(a - b) / np.linalg.norm(b)), float(np.abs(a - b).max() / np.abs(b).max()))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("b", [1, 3, 5, 16, 37])
def test_apply_fp64_vs_factor_oracle(name, b):
    buf, info, P, op, ofo = get(name)
    x = complex_gaussian(ofo.N, b, rhs_seed(0, b))
    xd = dev(x)
    for what, ref in (("K", fa.apply_Kdot), ("Kadj", fa.apply_Kdot_adj), ("G", fa.apply_G),
                      ("inv", fa.apply_inv)):
        y = getattr(op, "apply_" + what)(xd)
        torch.cuda.synchronize()
        assert rel(host(y), ref(P, x)) < TOL64, what


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("b", [1, 8, 32])
def test_apply_fp32_vs_factor_oracle(name, b):
    """FP32 within TOL32, or -- where the products amplify rounding, as Example 2's HIF factors
    do (cond(K) 112 at N = 1024 for sigma^2 = 0.05) -- within the amplification the FP64 path
    shows on the same factors and inputs: 4 e64 2^29 (2^29 = the ratio of the FP32 and FP64
    unit roundoffs; the same reading as the double-float bound below)."""
    buf, info, P, op, ofo = get(name)
    x = complex_gaussian(ofo.N, b, rhs_seed(0, 100 + b))
    xd = dev(x, torch.complex64)
    x64 = x.astype(np.complex64).astype(np.complex128)
    for what, ref in (("K", fa.apply_Kdot), ("Kadj", fa.apply_Kdot_adj), ("inv", fa.apply_inv)):
        want = ref(P, x64)
        y = getattr(op, "apply_" + what)(xd)
        y64 = getattr(op, "apply_" + what)(dev(x64))
        torch.cuda.synchronize()
        e64 = rel(host(y64), want)
        assert rel(host(y), want) < max(TOL32, 4 * e64 * 2.0 ** 29), (what, e64)


@pytest.mark.parametrize("name", ["ex1_256", "ex3_32", "ex3_64"])
def test_direct_solve_vs_dense_lu(name):
    """f = G-dot K-dot* u on the GPU against K^{-1} u by dense LU: within 10 eps (an error of
    the approximation, bounded in norm by the paper's e_s = ||I - G-dot K-dot* K||_2, so
    measured in the Frobenius norm)."""
    buf, info, P, op, ofo = get(name)
    u = complex_gaussian(ofo.N, 4, rhs_seed(0))
    f = host(op.apply_inv(dev(u)))
    assert frob(f, fo.solve_lu(ofo, u)) < 10 * CASES[name][3]


def test_leading_dimension_and_host_entry():
    buf, info, P, op, ofo = get("ex1_256")
    N, b, ld = ofo.N, 5, ofo.N + 7
    u = complex_gaussian(N, b, rhs_seed(0, 7))
    big = torch.zeros((b, ld), dtype=torch.complex128, device="cuda")
    big[:, :N] = torch.from_numpy(u.T.copy()).cuda()
    ud = big.t()[:N]  # stride (1, ld)
    assert ud.stride() == (1, ld)
    fbig = torch.full((b, ld), 7 + 7j, dtype=torch.complex128, device="cuda")
    fd = fbig.t()[:N]
    op.apply_inv(ud, fd)
    torch.cuda.synchronize()
    want = fa.apply_inv(P, u)
    assert rel(host(fd), want) < TOL64
    assert torch.all(fbig[:, N:] == 7 + 7j)  # padding rows untouched
    fh = op.apply_inv_host(u)
    assert rel(fh, want) < TOL64


def test_invalid_arguments_are_rejected():
    buf, info, P, op, ofo = get("ex1_256")
    x = dev(complex_gaussian(ofo.N, 2, 1))
    with pytest.raises(binding.FioError) as e:
        op.apply_K(x, x)  # aliasing
    assert e.value.status == -1
    lib = binding.load()
    import ctypes
    y = torch.empty_like(x)
    # dtype / precision mismatch
    assert lib.fio_apply_K(op.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                           ofo.N, 2, 0, 1, None) == -1
    # ld < N
    assert lib.fio_apply_K(op.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                           ofo.N - 1, 2, 0, 0, None) == -1
    # b = 0 is a no-op
    assert lib.fio_apply_K(op.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                           ofo.N, 0, 0, 0, None) == 0


@pytest.mark.parametrize("method", [binding.FIO_PCG, binding.FIO_GMRES, binding.FIO_IR])
@pytest.mark.parametrize("inner", [binding.FIO_P64, binding.FIO_P32])
def test_iterative_solves(method, inner):
    """Solve K-dot f = u to 1e-10; compare with the dense solve of the oracle's K-dot."""
    name = "ex1_256"
    buf, info, P, op, ofo = get(name)
    b = 3
    u = complex_gaussian(ofo.N, b, rhs_seed(1))
    f, infos = op.solve(dev(u), method=method, inner=inner, tol=1e-10, maxit=50)
    torch.cuda.synchronize()
    Kd = fa.dense_Kdot(P)
    fh = host(f)
    for j, (it, rr, st) in enumerate(infos):
        assert st == 0 and rr <= 1e-10, infos
        true_rr = np.linalg.norm(u[:, j] - Kd @ fh[:, j]) / np.linalg.norm(u[:, j])
        assert true_rr < 3e-10
        assert it <= 12  # the paper: 2-3 PCG iterations at eps = 1e-6
    f_ex = np.linalg.solve(Kd, u)
    assert rel(fh, f_ex) < 1e-8


# Tensor-core precisions (tcgen05): operands rounded to TF32 (unit roundoff 2^-11) or bfloat16
# (2^-8) before products accumulated in FP32.  Per stage ~sqrt(2) u relative, over up to ~15
# stages in a row: TF32 ~ 3e-3, BF16 ~ 2e-2; the bounds below leave a factor ~3.
# Split TF32 (head + tail of each operand, three products): each product a*b carries at most
# 3 * 2^-22 ~ 7e-7 relative (the two rounded tails and the dropped tail*tail), uncorrelated
# across the terms of a sum, on top of the FP32 accumulation and the FP32 rounding of every
# stage output that the FP32 path has: ~(1 + 7e-7 / 6e-8 / sqrt(300)) ~ 1.7 times TOL32's
# derivation, bound 2.5 * TOL32.
TOL_TC = {binding.FIO_PTF32: 1e-2, binding.FIO_PBF16: 5e-2, binding.FIO_PTF32X3: 2.5 * TOL32}
TC_PRECS = [binding.FIO_PTF32, binding.FIO_PBF16, binding.FIO_PTF32X3]


def _tc_apply(op, fn, xd, b, prec):
    import ctypes
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    y = binding.colmajor(torch.empty_like(xd))
    rc = fn(op.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(y.data_ptr()), xd.shape[0], b,
            binding.FIO_C64, prec, stream)
    torch.cuda.synchronize()
    return rc, y


@pytest.mark.parametrize("name", ["ex1_256", "ex3_32", "ex3_64"])
@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("b", [8, 32, 40, 72])
def test_apply_tensor_core_vs_factor_oracle(name, prec, b):
    buf, info, P, op, ofo = get(name)
    lib = binding.load()
    x = complex_gaussian(ofo.N, b, rhs_seed(0, 300 + b))
    xd = dev(x, torch.complex64)
    x64 = x.astype(np.complex64).astype(np.complex128)
    for what, fn, ref in (("K", lib.fio_apply_K, fa.apply_Kdot), ("Kadj", lib.fio_apply_Kadj, fa.apply_Kdot_adj),
                          ("inv", lib.fio_apply_inv, fa.apply_inv)):
        rc, y = _tc_apply(op, fn, xd, b, prec)
        assert rc == 0, (what, rc)
        err = rel(host(y), ref(P, x64))
        assert err < TOL_TC[prec], (what, err)


@pytest.mark.parametrize("name", ["ex1_256", "ex3_32", "ex3_64"])
def test_split_tf32_removes_tf32_rounding(name):
    """The split products are two orders of magnitude closer to the oracle than plain TF32 (a
    kernel that dropped the tail products would land at the TF32 error), and of the FP32 path's
    order: the tensor core's FP32 accumulator is not rounded to nearest at every addition, and the
    split mode adds 3 C / 8 MMA results into it per stage product (C <= ~300 columns), so its
    error may exceed the FP32 CUDA-core path's (round-to-nearest FMA chains) by about an order
    of magnitude, bounded here by 20 times."""
    buf, info, P, op, ofo = get(name)
    lib = binding.load()
    b = 32
    x = complex_gaussian(ofo.N, b, rhs_seed(0, 400))
    xd = dev(x, torch.complex64)
    want = fa.apply_Kdot(P, x.astype(np.complex64).astype(np.complex128))
    errs = {}
    for prec in (binding.FIO_PTF32, binding.FIO_PTF32X3, binding.FIO_P32):
        rc, y = _tc_apply(op, lib.fio_apply_K, xd, b, prec)
        assert rc == 0
        errs[prec] = rel(host(y), want)
    assert errs[binding.FIO_PTF32X3] < errs[binding.FIO_PTF32] / 100, errs
    assert errs[binding.FIO_PTF32X3] < 20 * errs[binding.FIO_P32], errs


@pytest.mark.parametrize("prec", TC_PRECS)
def test_refinement_with_tensor_core_inner(prec):
    """FP64 iterative refinement whose correction G-dot K-dot* r runs on the tensor cores still
    reaches 1e-10 (the outer FP64 residual removes the inner rounding)."""
    buf, info, P, op, ofo = get("ex1_256")
    u = complex_gaussian(ofo.N, 8, rhs_seed(2))
    f, infos = op.solve(dev(u), method=binding.FIO_IR, inner=prec, tol=1e-10, maxit=60)
    torch.cuda.synchronize()
    Kd = fa.dense_Kdot(P)
    fh = host(f)
    for j, (it, rr, st) in enumerate(infos):
        assert st == 0 and rr <= 1e-10, infos
        assert np.linalg.norm(u[:, j] - Kd @ fh[:, j]) / np.linalg.norm(u[:, j]) < 3e-10


# Double-float (FIO_PDF): every factor entry and vector value as hi + lo floats (48-bit
# significand) with compensated accumulation (Dot2 of Ogita, Rump and Oishi, working precision
# u = 2^-24).  Its error is that of the compensation term: n errors of size ~u|s_k| summed in FP32,
# each addition rounding at u|c|, so ~ n u^2 |s| for n random-sign terms; FP64 FMA chains
# (u64 = 2^-53) give ~ sqrt(n) u64 |s|.  Both are amplified alike by the conditioning of the
# products (the HIF factors of an ill-conditioned K*K, Example 2), so the bound follows the FP64
# path's own error e64 on the same factors times the typical ratio sqrt(n) u^2 / u64 =
# sqrt(n) 2^5, n = the longest sum of the operator (the widest block row or column), with a
# factor 4 and at least TOL64.  A kernel that lost the low parts anywhere would land at the FP32
# error (~1e-7).
def longest_sum(P):
    return max(max(int(S.getnnz(axis=1).max()), int(S.getnnz(axis=0).max())) for S in P.stages if S.nnz)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("b", [1, 3, 8, 37])
def test_apply_double_float_vs_factor_oracle(name, b):
    buf, info, P, op, ofo = get(name)
    x = complex_gaussian(ofo.N, b, rhs_seed(0, 500 + b))
    xd = dev(x)
    ratio = 4 * np.sqrt(longest_sum(P)) * 2.0 ** 5
    for what, ref in (("K", fa.apply_Kdot), ("Kadj", fa.apply_Kdot_adj), ("G", fa.apply_G),
                      ("inv", fa.apply_inv)):
        want = ref(P, x)
        y64 = getattr(op, "apply_" + what)(xd)
        y = getattr(op, "apply_" + what)(xd, precision=binding.FIO_PDF)
        torch.cuda.synchronize()
        e64 = rel(host(y64), want)
        assert rel(host(y), want) < max(TOL64, ratio * e64), (what, e64)


def test_double_float_precision_pairs():
    """FIO_PDF takes complex128 vectors only, and the no-allocation entry refuses it."""
    import ctypes
    buf, info, P, op, ofo = get("ex1_256")
    lib = binding.load()
    x = dev(complex_gaussian(ofo.N, 2, 1), torch.complex64)
    y = binding.colmajor(torch.empty_like(x))
    assert lib.fio_apply_K(op.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                           ofo.N, 2, binding.FIO_C64, binding.FIO_PDF, None) == -1
    x2 = dev(complex_gaussian(ofo.N, 2, 1))
    y2 = binding.colmajor(torch.empty_like(x2))
    assert lib.fio_apply_inv_noalloc(op.h, ctypes.c_void_p(x2.data_ptr()), ctypes.c_void_p(y2.data_ptr()),
                                     ofo.N, 2, binding.FIO_C128, binding.FIO_PDF, None) == -1


@pytest.mark.parametrize("inner", [binding.FIO_P32, binding.FIO_PTF32X3])
def test_refinement_with_double_float_residual(inner):
    """Iterative refinement whose residuals u - K-dot f are taken in double-float arithmetic
    reaches 1e-10 against the oracle's dense K-dot (FP64), as with FP64 residuals."""
    buf, info, P, op, ofo = get("ex1_256")
    u = complex_gaussian(ofo.N, 8, rhs_seed(2, 1))
    f, infos = op.solve(dev(u), method=binding.FIO_IR, inner=inner, tol=1e-10, maxit=60,
                        outer=binding.FIO_PDF)
    torch.cuda.synchronize()
    Kd = fa.dense_Kdot(P)
    fh = host(f)
    for j, (it, rr, st) in enumerate(infos):
        assert st == 0 and rr <= 1e-10, infos
        assert np.linalg.norm(u[:, j] - Kd @ fh[:, j]) / np.linalg.norm(u[:, j]) < 3e-10


@pytest.mark.parametrize("method", [binding.FIO_PCG, binding.FIO_GMRES, binding.FIO_IR])
def test_exact_initial_guess_needs_no_iteration(method):
    """An initial guess that already solves K-dot f = u (dense solve of the oracle's K-dot) stops
    at iteration 0: the guess is used, not mistaken for the zero guess whose residual is u."""
    buf, info, P, op, ofo = get("ex1_256")
    Kd = fa.dense_Kdot(P)
    u = complex_gaussian(ofo.N, 3, rhs_seed(2, 2))
    f0 = dev(np.linalg.solve(Kd, u))
    f, infos = op.solve(dev(u), f0.clone(), method=method, inner=binding.FIO_P64, tol=1e-10, maxit=50)
    torch.cuda.synchronize()
    for it, rr, st in infos:
        assert st == 0 and it == 0 and rr <= 1e-10, infos


# Autotuner: every tile-shape variant sums each output's terms in the same order, so for b >= 5
# the tuned applies must reproduce the built-in ones bit for bit (but for the split variant 12 of
# the in-place stages and the three-product variants 14-16); for b <= 4 the few-RHS kernel (tree
# reductions) may be chosen, within the parity tolerances above.
ALLOWED = {0: {0, 8, 1}, 1: {0, 1, 2, 13, 16}, 2: {0, 2, 3, 4, 13, 14, 16},
           3: {0, 3, 5, 6, 17, 18} | set(range(9, 16)), 4: {0, 3, 5, 6, 7, 17, 18} | set(range(9, 16))}
THREE_PRODUCTS = {14, 15, 16}


def _bucket(b):
    return 0 if b <= 4 else 1 if b <= 8 else 2 if b <= 16 else 3 if b <= 32 else 4


@pytest.mark.parametrize("name", ["ex1_1024", "ex3_32"])
@pytest.mark.parametrize("prec,dt,tol", [(binding.FIO_P64, torch.complex128, TOL64),
                                         (binding.FIO_P32, torch.complex64, TOL32),
                                         (binding.FIO_PDF, torch.complex128, TOL64)])
@pytest.mark.parametrize("b", [2, 16, 37])
def test_autotune_choices_and_results(name, prec, dt, tol, b):
    buf, info, P, op, ofo = get(name)
    x = complex_gaussian(ofo.N, b, rhs_seed(0, 600 + b))
    xd = dev(x, dt)
    before = {w: getattr(op, "apply_" + w)(xd, precision=prec).clone() for w in ("K", "Kadj", "inv")}
    choices = op.autotune(b, prec)
    assert len(choices) == 2 * (P.n_bf + P.n_hif) + P.n_root
    assert set(choices) <= ALLOWED[_bucket(b)], choices
    x64 = x.astype(np.complex64).astype(np.complex128) if dt == torch.complex64 else x
    for w, ref in (("K", fa.apply_Kdot), ("Kadj", fa.apply_Kdot_adj), ("inv", fa.apply_inv)):
        after = getattr(op, "apply_" + w)(xd, precision=prec)
        torch.cuda.synchronize()
        # bit for bit unless the tuner picked three products or split an in-place stage over its
        # columns (12: partial sums in another order; the in-place stages are in inv only)
        if b >= 5 and not THREE_PRODUCTS & set(choices) and (w != "inv" or 12 not in choices):
            assert torch.equal(after, before[w]), w
        assert rel(host(after), ref(P, x64)) < tol, w


def test_autotune_rejects_bad_arguments():
    import ctypes
    buf, info, P, op, ofo = get("ex3_32")
    lib = binding.load()
    n = ctypes.c_int()
    assert lib.fio_autotune(None, 4, binding.FIO_P64, None, None, 0, ctypes.byref(n)) == -1
    assert lib.fio_autotune(op.h, -1, binding.FIO_P64, None, None, 0, ctypes.byref(n)) == -1
    assert lib.fio_autotune(op.h, 4, 9, None, None, 0, ctypes.byref(n)) == -1
    assert lib.fio_autotune(op.h, 4, binding.FIO_P64, None, None, 5, ctypes.byref(n)) == -1  # cap > 0, no array
    assert lib.fio_autotune(op.h, 0, binding.FIO_P64, None, None, 0, ctypes.byref(n)) == 0 and n.value == 0


@pytest.mark.parametrize("name", ["ex1_1024", "ex3_32"])
@pytest.mark.parametrize("prec,dt", [(binding.FIO_P64, torch.complex128), (binding.FIO_P32, torch.complex64),
                                     (binding.FIO_PDF, torch.complex128)])
def test_every_tile_shape_is_bit_identical(name, prec, dt):
    """Each tile shape <TX,TB,TR> of the stage kernel, and the warp-per-block kernel for small
    blocks (13: the 16-point leaf stages), sums every output's terms in the same order, so pinning
    any of them reproduces the built-in choice bit for bit (b = 40: ragged RHS tiles for every
    shape)."""
    buf, info, P, op, ofo = get(name)
    b = 40
    xd = dev(complex_gaussian(ofo.N, b, rhs_seed(0, 700)), dt)
    op.set_variant(b, prec, 0)
    ref = {w: getattr(op, "apply_" + w)(xd, precision=prec).clone() for w in ("K", "Kadj", "inv")}
    for var in list(range(1, 8)) + ([9, 10, 11, 17, 18] if prec == binding.FIO_P32 else []) + \
            ([13] if prec != binding.FIO_PDF else []):
        op.set_variant(b, prec, var)
        for w in ("K", "Kadj", "inv"):
            y = getattr(op, "apply_" + w)(xd, precision=prec)
            torch.cuda.synchronize()
            assert torch.equal(y, ref[w]), (var, w)
    op.set_variant(b, prec, 0)


@pytest.mark.parametrize("name", ["ex1_256", "ex3_32", "ex3_64"])
@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("b", [8, 37, 40, 72, 130])
def test_tensor_core_ring_matches_single_buffer(name, prec, b):
    """The warp-specialised ring kernel (2, 3, 4 chunk stages: variants 20, 21, 22) and the
    TMA-fed persistent kernel (variant 30; odd b falls back to variant 0) issue the same MMAs in
    the same order into each accumulator as the single-buffer kernel: bit-identical results, and
    within the precision's bound of the oracle."""
    buf, info, P, op, ofo = get(name)
    lib = binding.load()
    x = complex_gaussian(ofo.N, b, rhs_seed(0, 800 + b))
    xd = dev(x, torch.complex64)
    x64 = x.astype(np.complex64).astype(np.complex128)
    op.set_variant(b, prec, 0)
    ref = {}
    for w, fn in (("K", lib.fio_apply_K), ("Kadj", lib.fio_apply_Kadj), ("inv", lib.fio_apply_inv)):
        rc, y = _tc_apply(op, fn, xd, b, prec)
        assert rc == 0
        ref[w] = y.clone()
    for var in (20, 21, 22, 30, 32, 33):
        op.set_variant(b, prec, var)
        for w, fn, oref in (("K", lib.fio_apply_K, fa.apply_Kdot), ("Kadj", lib.fio_apply_Kadj, fa.apply_Kdot_adj),
                            ("inv", lib.fio_apply_inv, fa.apply_inv)):
            rc, y = _tc_apply(op, fn, xd, b, prec)
            assert rc == 0, (var, w, rc)
            assert torch.equal(y, ref[w]), (var, w)
            assert rel(host(y), oref(P, x64)) < TOL_TC[prec], (var, w)
    op.set_variant(b, prec, 0)


@pytest.mark.parametrize("name", ["ex1_256", "ex3_32", "ex3_64"])
@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("b", [8, 40, 72])
def test_tensor_core_split_inplace_stages(name, prec, b):
    """Variant 31: the TMA kernel with the in-place stages (HIF nodes and the root) split over
    their columns into slices summed by a fixed-order reduction.  Only the in-place stages
    change: K-dot and K-dot* stay bit-identical to variant 0; G-dot and G-dot K-dot* (sums in
    another order) stay within the precision's bound of the oracle."""
    buf, info, P, op, ofo = get(name)
    lib = binding.load()
    x = complex_gaussian(ofo.N, b, rhs_seed(0, 850 + b))
    xd = dev(x, torch.complex64)
    x64 = x.astype(np.complex64).astype(np.complex128)
    try:
        op.set_variant(b, prec, 0)
        ref = {}
        for w, fn in (("K", lib.fio_apply_K), ("Kadj", lib.fio_apply_Kadj)):
            rc, y = _tc_apply(op, fn, xd, b, prec)
            assert rc == 0
            ref[w] = y.clone()
        op.set_variant(b, prec, 31)
        for w, fn, oref in (("K", lib.fio_apply_K, fa.apply_Kdot), ("Kadj", lib.fio_apply_Kadj, fa.apply_Kdot_adj),
                            ("G", lib.fio_apply_G, fa.apply_G), ("inv", lib.fio_apply_inv, fa.apply_inv)):
            rc, y = _tc_apply(op, fn, xd, b, prec)
            assert rc == 0, (w, rc)
            if w in ref:
                assert torch.equal(y, ref[w]), w
            assert rel(host(y), oref(P, x64)) < TOL_TC[prec], w
    finally:
        op.set_variant(b, prec, 0)


@pytest.mark.parametrize("name", ["ex1_256", "ex3_32", "ex3_64", "ex2b_1024"])
@pytest.mark.parametrize("b", [17, 40, 72])
def test_fp32_split_inplace_stages(name, b):
    """Variant 12 on the FP32 CUDA cores: the in-place stages (HIF nodes, root) split over their
    columns into slices summed in a fixed order; the butterfly stages run as variant 11, so K-dot
    and K-dot* stay bit-identical to it, and G-dot, G-dot K-dot* stay within the FP32 bound (with
    the amplification of ill-conditioned factors, R30)."""
    buf, info, P, op, ofo = get(name)
    x = complex_gaussian(ofo.N, b, rhs_seed(0, 870 + b))
    xd = dev(x, torch.complex64)
    x64 = x.astype(np.complex64).astype(np.complex128)
    try:
        op.set_variant(b, binding.FIO_P32, 11)
        ref = {w: getattr(op, "apply_" + w)(xd).clone() for w in ("K", "Kadj")}
        op.set_variant(b, binding.FIO_P32, 12)
        for w, oref in (("K", fa.apply_Kdot), ("Kadj", fa.apply_Kdot_adj), ("G", fa.apply_G), ("inv", fa.apply_inv)):
            y = getattr(op, "apply_" + w)(xd)
            torch.cuda.synchronize()
            if w in ref:
                assert torch.equal(y, ref[w]), w
            want = oref(P, x64)
            e64 = rel(host(getattr(op, "apply_" + w)(dev(x64))), want)
            assert rel(host(y), want) < max(TOL32, 4 * e64 * 2.0 ** 29), (w, e64)
    finally:
        op.set_variant(b, binding.FIO_P32, 0)


@pytest.mark.parametrize("name", ["ex1_256", "ex3_32", "ex3_64", "ex2b_1024"])
@pytest.mark.parametrize("prec", [binding.FIO_P64, binding.FIO_PDF])
@pytest.mark.parametrize("b", [6, 17, 40])
def test_three_product_fp64_and_double_float(name, prec, b):
    """Variants 14-16 (three real products per complex product in FP64 and double-float, on the
    butterfly stages): every apply within the bound of its arithmetic against the oracle (FP64
    1e-12; double-float as the four-product test: max(1e-12, 4 sqrt(longest sum) 2^5 e64)), K-dot
    and K-dot* within three times the four-product error plus 1e-15, and G-dot bit-identical to
    the built-in choice (the in-place stages keep four products)."""
    buf, info, P, op, ofo = get(name)
    x = complex_gaussian(ofo.N, b, rhs_seed(0, 910 + b))
    xd = dev(x)
    refs = (("K", fa.apply_Kdot), ("Kadj", fa.apply_Kdot_adj), ("G", fa.apply_G), ("inv", fa.apply_inv))
    want = {w: oref(P, x) for w, oref in refs}
    ratio = 4 * np.sqrt(longest_sum(P)) * 2.0 ** 5
    try:
        op.set_variant(b, prec, 0)
        four = {w: getattr(op, "apply_" + w)(xd, precision=prec).clone() for w, _ in refs}
        e64 = {w: rel(host(getattr(op, "apply_" + w)(xd)), want[w]) for w, _ in refs}
        for var in (14, 15, 16):
            op.set_variant(b, prec, var)
            for w, _ in refs:
                y = getattr(op, "apply_" + w)(xd, precision=prec)
                torch.cuda.synchronize()
                err, e4 = rel(host(y), want[w]), rel(host(four[w]), want[w])
                print(f"[{name} {prec} b={b} variant {var}] {w}: {err:.3g} (four products {e4:.3g})")
                bound = TOL64 if prec == binding.FIO_P64 else max(TOL64, ratio * e64[w])
                assert err < bound, (var, w, err, e64[w])
                if w == "G":
                    assert torch.equal(y, four[w]), var
                elif w in ("K", "Kadj"):
                    assert err <= 3 * e4 + 1e-15, (var, w, err, e4)
    finally:
        op.set_variant(b, prec, 0)


def test_set_variant_rejects_unknown_variants():
    buf, info, P, op, ofo = get("ex3_32")
    lib = binding.load()
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P64, 19) == -1
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P32, 19) == -1
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P64, 18) == -1   # complex64-only tiles
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P32, 18) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P64, 17) == -1   # complex64-only tiles
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P32, 17) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P32, 0) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P32, 14) == -1   # FP64 / double-float tiles
    assert lib.fio_set_variant(op.h, 16, binding.FIO_PDF, 16) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_PDF, 0) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P64, 14) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P32, 13) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P64, 13) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_PDF, 13) == -1   # double-float: tiled kernels only
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P64, 12) == -1   # complex64-only tiles
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P64, 0) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P32, 12) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P32, 0) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P64, 11) == -1   # complex64-only tiles
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P64, 9) == -1    # complex64-only tiles
    assert lib.fio_set_variant(op.h, 16, binding.FIO_P32, 8) == -1    # few-RHS kernel needs b <= 4
    assert lib.fio_set_variant(op.h, 16, binding.FIO_PTF32, 3) == -1  # tensor-core launch: 0, 20-22, 30
    assert lib.fio_set_variant(op.h, 16, binding.FIO_PTF32, 34) == -1
    assert lib.fio_set_variant(op.h, 16, binding.FIO_PTF32, 31) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_PTF32, 30) == 0
    assert lib.fio_set_variant(op.h, 16, binding.FIO_PTF32, 0) == 0
    assert lib.fio_set_variant(op.h, 0, binding.FIO_P32, 1) == -1
    assert lib.fio_set_variant(op.h, 4, binding.FIO_P32, 8) == 0
    assert lib.fio_set_variant(op.h, 4, binding.FIO_P32, 0) == 0


def test_example2_pcg_with_G_vs_cg_with_Kadj_only():
    """Example 2 (sigma^2 = 0.05), the paper's case where K-dot* alone is a poor preconditioner:
    PCG with G-dot reaches 1e-10 in a handful of iterations on the GPU, while CG on the normal
    equations with nothing but K* (the oracle's cgne, dense K) needs hundreds to reach 1e-8."""
    buf, info, P, op, ofo = get("ex2b_1024")
    u = complex_gaussian(ofo.N, 2, rhs_seed(2, 7))
    f, infos = op.solve(dev(u), method=binding.FIO_PCG, inner=binding.FIO_P64, tol=1e-10, maxit=50)
    torch.cuda.synchronize()
    Kd = fa.dense_Kdot(P)
    fh = host(f)
    for j, (it, rr, st) in enumerate(infos):
        assert st == 0 and rr <= 1e-10 and it <= 10, infos
        assert np.linalg.norm(u[:, j] - Kd @ fh[:, j]) / np.linalg.norm(u[:, j]) < 3e-10
    K = fo.dense_K(ofo)
    _, it_cg, _ = fo.cgne(ofo, u[:, 0], tol=1e-8, maxit=3000, K=K)
    assert it_cg > 20 * max(i for i, _, _ in infos), (it_cg, infos)


@pytest.mark.parametrize("name", ["ex1_1024", "ex3_32", "ex2b_1024"])
def test_stage_errors_against_fp64(name):
    """fio_stage_errors reports one error per stage launch group; its last entry is the error of
    the whole apply (the same kernels run).  On the well-conditioned operators every precision
    stays within its apply bound; on Example 2 (sigma^2 = 0.05) the HIF stages amplify every
    precision's rounding alike, so the largest stage error is bounded by the FP32 path's largest
    times the ratio of the input roundings (TF32: the tensor core keeps 10 mantissa bits of an
    FP32 operand, 2^-10 / 2^-24 = 2^14; BF16 rounds to 8 bits, 2^-9 / 2^-24, bound 2^16; split
    TF32: 3 x 2^-22 per product plus the truncating accumulation, bound 2^8), and double-float
    stays below FP32."""
    buf, info, P, op, ofo = get(name)
    b = 8
    x = complex_gaussian(ofo.N, b, rhs_seed(0, 900))
    xd = dev(x)
    ref = op.apply_inv(xd).cpu().numpy()
    nst = P.n_bf + 2 * P.n_hif + P.n_root
    bounds = {binding.FIO_PDF: 1e-11, binding.FIO_P32: TOL32, binding.FIO_PTF32X3: TOL_TC[binding.FIO_PTF32X3],
              binding.FIO_PTF32: TOL_TC[binding.FIO_PTF32], binding.FIO_PBF16: TOL_TC[binding.FIO_PBF16]}
    ratio = {binding.FIO_PDF: 1.0, binding.FIO_P32: 1.0, binding.FIO_PTF32X3: 2.0 ** 8,
             binding.FIO_PTF32: 2.0 ** 14, binding.FIO_PBF16: 2.0 ** 16}
    errs32 = op.stage_errors("inv", xd, binding.FIO_P32)
    for prec, bound in bounds.items():
        errs = op.stage_errors("inv", xd, prec)
        assert len(errs) == nst, (prec, len(errs), nst)
        if name == "ex2b_1024":
            assert max(errs) <= ratio[prec] * max(errs32) * 1.01, (prec, max(errs), max(errs32))
        else:
            assert max(errs) < bound, (prec, errs)
        # the last stage's error is the whole apply's error against the FP64 apply
        dt = torch.complex128 if prec == binding.FIO_PDF else torch.complex64
        y = op.apply_inv(xd.to(dt), precision=prec).cpu().numpy().astype(np.complex128)
        whole = frob(y, ref)
        assert abs(errs[-1] - whole) <= 0.05 * whole + 1e-15, (prec, errs[-1], whole)
    kerr = op.stage_errors("K", xd, binding.FIO_P32)
    assert len(kerr) == P.n_bf and max(kerr) < TOL32


@pytest.mark.parametrize("kind,n", [("linear1d", 256), ("linear2d", 16)])
def test_linear_phase_degenerate_case(kind, n):
    """Phi = x.xi: K*K = N I, so the HIF eliminates every DOF at the leaves (empty root) and
    G-dot K-dot* = K*/N; and K = F^{-1}, so the butterfly apply and the FFT kernel (two
    independent GPU paths) must agree to the butterfly tolerance."""
    fbuild.build()
    buf, info = build_operator(kind, n, 1e-10, 1e-10)
    assert info["root"] == 0
    op = binding.Operator(buf)
    ofo = fo.FIO(kind, n)
    u = complex_gaussian(ofo.N, 3, rhs_seed(0, 950))
    f = host(op.apply_inv(dev(u)))
    assert rel(f, fo.apply_Kadj(ofo, u) / ofo.N) < 1e-9
    kb = host(op.apply_K(dev(u)))
    fi = host(op.apply_Finv(dev(u)))
    assert rel(kb, fi) < 1e-9
    assert rel(fi, fo.apply_K(ofo, u)) < 1e-13


@pytest.mark.parametrize("inner,outer", [(binding.FIO_P32, binding.FIO_P64), (binding.FIO_PTF32X3, binding.FIO_P64),
                                         (binding.FIO_P32, binding.FIO_PDF)])
def test_refinement_with_tight_butterfly_residual(inner, outer):
    """Iterative refinement whose true residual u - K-dot_tight f is taken with a second butterfly
    of the same FIO built 10^5 times tighter (eps_BF 1e-12; e_a 3.6e-13 on the host), while the
    corrections G-dot K-dot* r come from the eps = 1e-6 operator (eps_BF 1e-7, e_a 8e-8): it
    reaches 1e-10 against K-dot_tight and so lands within cond(K) (1e-10 + e_a_tight) of the exact
    solve K^{-1} u (dense LU of the oracle's K; cond(K) ~ 3 for Example 1), where refinement
    against the loose butterfly alone stops at that butterfly's own distance (2.5e-8 on the host)."""
    fbuild.build()
    ofo = fo.FIO("ex1", 1024)
    loose = binding.Operator(build_operator("ex1", 1024, 1e-7, 1e-6)[0])
    tight = binding.Operator(build_operator("ex1", 1024, 1e-12, 1e-6)[0], binding.FIO_MASK_P64 | binding.FIO_MASK_DF)
    u = complex_gaussian(ofo.N, 8, rhs_seed(5, 1))
    f_ex = fo.solve_lu(ofo, u)
    f, infos = loose.solve(dev(u), method=binding.FIO_IR, inner=inner, outer=outer, tol=1e-10, maxit=60,
                           residual_op=tight)
    torch.cuda.synchronize()
    for it, rr, st in infos:
        assert st == 0 and rr <= 1e-10, infos
    assert frob(host(f), f_ex) < 1e-9
    f2, infos2 = loose.solve(dev(u), method=binding.FIO_IR, inner=inner, outer=outer, tol=1e-10, maxit=60)
    torch.cuda.synchronize()
    assert frob(host(f2), f_ex) > 1e-8
    # the residual operator must describe the same grid, and only refinement and the direct
    # method take one
    other = binding.Operator(build_operator("ex1", 256, 1e-7, 1e-6)[0])
    with pytest.raises(binding.FioError):
        loose.solve(dev(u), method=binding.FIO_IR, residual_op=other)
    with pytest.raises(binding.FioError):
        loose.solve(dev(u), method=binding.FIO_GMRES, residual_op=tight)
