"""fio_apply_inv_noalloc: the direct solve for callers that may not allocate device memory while
they run (their memory belongs to another allocator, or the implicit synchronisation of
cudaMalloc is unacceptable in their loop).  Its scratch is a static device array, so the call must
give the same answer as fio_apply_inv, call after call, with whatever the previous call left in
that array.  The same stage kernels run in the same order on both entry points, so the results
are compared bit for bit, in every precision the entry point accepts, and against the oracle's
product of the same factors.  This file is collected last so that a run stopping at the first
failure has already run every other test."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import factor_apply as fa  # noqa: E402
from paper_2105_02995_gb300 import binding, build as fbuild  # noqa: E402
from paper_2105_02995_gb300.builder import build_operator  # noqa: E402
from paper_2105_02995_gb300.inputs import complex_gaussian, rhs_seed  # noqa: E402

# precision -> (vector dtype, bound against the oracle's FP64 product of the same factors);
# the bounds are those of the parity tests (FP64 1e-12, FP32 2e-5, TF32 1e-2, BF16 5e-2, split
# TF32 2.5 x the FP32 bound)
PRECS = {
    binding.FIO_P64: (torch.complex128, 1e-12),
    binding.FIO_P32: (torch.complex64, 2e-5),
    binding.FIO_PTF32: (torch.complex64, 1e-2),
    binding.FIO_PBF16: (torch.complex64, 5e-2),
    binding.FIO_PTF32X3: (torch.complex64, 5e-5),
}
_op = {}


def _operator():
    if "op" not in _op:
        fbuild.build()
        buf, _ = build_operator("ex1", 256, 1e-7, 1e-6)
        _op["op"] = (binding.Operator(buf), fa.PackedFactors(buf))
    return _op["op"]


def _noalloc(lib, op, u, f, b, prec):
    dt = binding.FIO_C128 if u.dtype == torch.complex128 else binding.FIO_C64
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.fio_apply_inv_noalloc(op.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                     op.N, b, dt, prec, stream)


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("b", [2, 5, 32])
def test_noalloc_matches_allocating_entry_point(prec, b):
    """Two calls in a row (the second sees the first one's leftovers in the static array): each
    equals fio_apply_inv in the same precision bit for bit, and the oracle within the bound."""
    lib = binding.load()
    op, P = _operator()
    dtype, tol = PRECS[prec]
    N = op.N
    for call in range(2):
        u_np = complex_gaussian(N, b, rhs_seed(9, 10 * b + call))
        u = binding.colmajor(torch.from_numpy(u_np).to("cuda", dtype))
        want = op.apply_inv(u, precision=prec).clone()
        f = binding.colmajor(torch.full((N, b), 3.0 - 1.0j, dtype=dtype, device="cuda"))
        rc = _noalloc(lib, op, u, f, b, prec)
        assert rc == 0, binding.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        assert torch.equal(f, want), (prec, b, call)
        ref = fa.apply_inv(P, u.cpu().numpy().astype(np.complex128))
        got = f.cpu().numpy().astype(np.complex128)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < tol, (prec, b, call, err)


def test_noalloc_runs_the_tensor_cores():
    """With 8 or more right-hand sides the tensor-core precisions really run on the tensor cores:
    the TF32 result differs from the FP32 CUDA-core result by the TF32 rounding (~1e-3), far
    above the FP32 rounding; split TF32 lands between the two."""
    lib = binding.load()
    op, P = _operator()
    N, b = op.N, 32
    u = binding.colmajor(torch.from_numpy(complex_gaussian(N, b, rhs_seed(9, 99))).to("cuda", torch.complex64))
    out = {}
    for prec in (binding.FIO_P32, binding.FIO_PTF32, binding.FIO_PTF32X3):
        f = binding.colmajor(torch.empty((N, b), dtype=torch.complex64, device="cuda"))
        assert _noalloc(lib, op, u, f, b, prec) == 0
        torch.cuda.synchronize()
        out[prec] = f.clone()

    def d(p):
        return float(torch.linalg.norm(out[p] - out[binding.FIO_P32]) / torch.linalg.norm(out[binding.FIO_P32]))
    assert d(binding.FIO_PTF32) > 1e-4, d(binding.FIO_PTF32)
    assert 0 < d(binding.FIO_PTF32X3) < d(binding.FIO_PTF32) / 30, (d(binding.FIO_PTF32X3), d(binding.FIO_PTF32))


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    """A batch whose work vectors exceed the static array is refused (FIO_EINVAL) and nothing is
    written; a batch that fits still runs."""
    lib = binding.load()
    op, P = _operator()
    N = op.N
    # three work vectors of at least N x b complex128 each: b = 8192 needs >= 3 x 33.5 MB > 64 MiB
    b = 8192
    u = binding.colmajor(torch.ones((N, b), dtype=torch.complex128, device="cuda"))
    f = binding.colmajor(torch.full((N, b), 5.0 + 0j, dtype=torch.complex128, device="cuda"))
    rc = _noalloc(lib, op, u, f, b, binding.FIO_P64)
    assert rc == -1  # FIO_EINVAL
    torch.cuda.synchronize()
    assert torch.all(f == 5.0)
    rc = _noalloc(lib, op, u[:, :64], f[:, :64], 64, binding.FIO_P64)
    assert rc == 0
    torch.cuda.synchronize()
