"""fio_apply_inv_noalloc: the direct solve for callers that may not allocate device memory while
they run (their memory belongs to another allocator, or the implicit synchronisation of
cudaMalloc is unacceptable in their loop).  Its scratch is a static device array, so the call must
give the same answer as fio_apply_inv, call after call, with whatever the previous call left in
that array.  This file is collected last so that a run stopping at the first failure has already
run every other test."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2105_02995_gb300 import binding, build as fbuild  # noqa: E402
from paper_2105_02995_gb300.builder import build_operator  # noqa: E402
from paper_2105_02995_gb300.inputs import complex_gaussian, rhs_seed  # noqa: E402


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 2e-5)])
def test_noalloc_matches_allocating_entry_point(dtype, tol):
    fbuild.build()
    lib = binding.load()
    buf, _ = build_operator("ex1", 256, 1e-7, 1e-6)
    op = binding.Operator(buf)
    N, b = op.N, 5
    dt, prec = (binding.FIO_C128, binding.FIO_P64) if dtype == torch.complex128 else (binding.FIO_C64, binding.FIO_P32)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        u = binding.colmajor(torch.from_numpy(complex_gaussian(N, b, rhs_seed(9, call))).to("cuda", dtype))
        want = op.apply_inv(u)
        f = binding.colmajor(torch.full((N, b), 3.0 - 1.0j, dtype=dtype, device="cuda"))
        rc = lib.fio_apply_inv_noalloc(op.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                       N, b, dt, prec, stream)
        assert rc == 0, binding.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        assert _rel(f, want) <= tol, (call, _rel(f, want))
    op.release()


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    """A batch whose work vectors exceed the static array is refused (FIO_EINVAL) and nothing is
    written; a batch that fits still runs."""
    lib = binding.load()
    buf, _ = build_operator("ex1", 256, 1e-7, 1e-6)
    op = binding.Operator(buf)
    N = op.N
    # three work vectors of at least N x b complex128 each: b = 8192 needs >= 3 x 33.5 MB > 64 MiB
    b = 8192
    u = binding.colmajor(torch.ones((N, b), dtype=torch.complex128, device="cuda"))
    f = binding.colmajor(torch.full((N, b), 5.0 + 0j, dtype=torch.complex128, device="cuda"))
    rc = lib.fio_apply_inv_noalloc(op.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                   N, b, binding.FIO_C128, binding.FIO_P64, None)
    assert rc == -1  # FIO_EINVAL
    torch.cuda.synchronize()
    assert torch.all(f == 5.0)
    rc = lib.fio_apply_inv_noalloc(op.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                   N, 64, binding.FIO_C128, binding.FIO_P64, None)
    assert rc == 0
    torch.cuda.synchronize()
    op.release()
