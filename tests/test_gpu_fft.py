"""The DFT F of section 1 and its inverse on the GPU (fio_apply_F / fio_apply_Finv) against the
oracle (oracle/fio_oracle.py: numpy.fft path, itself pinned to the dense definition), and the
full solve of u = K F f.

Sizes: 1D N = 256 and 2048 (one pass), 4096 and 65536 (four-step); 2D n = 8, 64, 256 (two passes);
ragged batches.  Bounds: an FFT of length N carries ~log2(N) roundings per value, so FP64 within
1e-13 and FP32 (with single-precision twiddles) within 5e-6 relative.
The operators here are minimal (one identity stage on the right grid): F depends only on n and d.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fio_oracle as fo  # noqa: E402
from paper_2105_02995_gb300 import binding, build as fbuild  # noqa: E402
from paper_2105_02995_gb300.builder.pack import pack  # noqa: E402
from paper_2105_02995_gb300.builder.stages import KIND_MAP, Stage  # noqa: E402
from paper_2105_02995_gb300.inputs import complex_gaussian, rhs_seed  # noqa: E402

_ops = {}


def grid_op(n, d):
    """An operator on the n^d grid whose only stage is the identity (16 x 16 blocks)."""
    key = (n, d)
    if key not in _ops:
        fbuild.build()
        N = n ** d
        st = Stage(KIND_MAP, N, N)
        eye = np.eye(16)
        for i in range(N // 16):
            st.add(eye, np.arange(16 * i, 16 * i + 16), np.arange(16 * i, 16 * i + 16))
        _ops[key] = binding.Operator(pack(d, n, [st], [], [], 0.0, 0.0))
    return _ops[key]


def dev(a, dtype):
    return binding.colmajor(torch.from_numpy(np.asarray(a)).to("cuda", dtype))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [(256, 1, 3), (2048, 1, 2), (4096, 1, 5), (65536, 1, 2), (8, 2, 3), (64, 2, 4), (256, 2, 2)]


@pytest.mark.parametrize("n,d,b", CASES)
@pytest.mark.parametrize("dt,tol", [(torch.complex128, 1e-13), (torch.complex64, 5e-6)])
def test_dft_vs_oracle(n, d, b, dt, tol):
    op = grid_op(n, d)
    x = complex_gaussian(n ** d, b, rhs_seed(6, n + b))
    xr = x.astype(np.complex64).astype(np.complex128) if dt == torch.complex64 else x
    xd = dev(x, dt)
    fh = op.apply_F(xd).cpu().numpy().astype(np.complex128)
    assert rel(fh, fo.apply_F(n, d, xr)) < tol
    fi = op.apply_Finv(xd).cpu().numpy().astype(np.complex128)
    assert rel(fi, fo.apply_Finv(n, d, xr)) < tol
    # round trip
    back = op.apply_Finv(op.apply_F(xd)).cpu().numpy().astype(np.complex128)
    assert rel(back, xr) < 2 * tol


def test_dft_leading_dimension_and_arguments():
    import ctypes
    op = grid_op(64, 2)
    N, b, ld = 4096, 3, 4096 + 5
    x = complex_gaussian(N, b, rhs_seed(6, 1))
    big = torch.zeros((b, ld), dtype=torch.complex128, device="cuda")
    big[:, :N] = torch.from_numpy(x.T.copy()).cuda()
    xd = big.t()[:N]
    ybig = torch.full((b, ld), 3 + 3j, dtype=torch.complex128, device="cuda")
    yd = ybig.t()[:N]
    op.apply_Finv(xd, yd)
    torch.cuda.synchronize()
    assert rel(yd.cpu().numpy(), fo.apply_Finv(64, 2, x)) < 1e-13
    assert torch.all(ybig[:, N:] == 3 + 3j)
    lib = binding.load()
    p = ctypes.c_void_p
    assert lib.fio_apply_Finv(op.h, p(xd.data_ptr()), p(xd.data_ptr()), ld, b, 0, 0, None) == -1  # aliasing
    assert lib.fio_apply_Finv(op.h, p(xd.data_ptr()), p(yd.data_ptr()), ld, b, 0, 1, None) == -1  # dtype/precision
    assert lib.fio_apply_F(op.h, p(xd.data_ptr()), p(yd.data_ptr()), N - 1, b, 0, 0, None) == -1  # ld < N


def test_full_solve_of_u_equals_K_F_f():
    """f = F^{-1} (G-dot K-dot* u) against the oracle's F^{-1} K^{-1} u (dense LU): within 10 eps,
    as for the direct solve (F^{-1} is n^{d/2} times unitary, so it keeps relative errors)."""
    from paper_2105_02995_gb300.builder import build_operator
    fbuild.build()
    n, eps = 256, 1e-6
    buf, info = build_operator("ex1", n, 1e-7, eps)
    op = binding.Operator(buf)
    ofo = fo.FIO("ex1", n)
    u = complex_gaussian(n, 4, rhs_seed(6, 2))
    fd = op.apply_Finv(op.apply_inv(dev(u, torch.complex128))).cpu().numpy()
    want = fo.apply_Finv(n, 1, fo.solve_lu(ofo, u))
    assert rel(fd, want) < 10 * eps
    # and the forward model reproduces u: K F f = u up to the same error
    assert rel(fo.apply_K(ofo, fo.apply_F(n, 1, fd)), u) < 10 * eps
