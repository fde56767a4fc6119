"""Failure paths on the GPU, tested without faulting or hanging the device.

* Bounded waits: fio_selftest_wait makes CTAs wait on an mbarrier that nothing arrives at, with a
  short limit; every wait must give up, the status must come back as FIO_ETIMEOUT, and the device
  must stay usable (an apply right after still matches the oracle).
* Non-convergence: an iterative solve capped below the iterations it needs returns FIO_ENOCONV
  with per-right-hand-side records.
* Bad solver options are refused before any launch.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import factor_apply as fa  # noqa: E402
from paper_2105_02995_gb300 import binding, build as fbuild  # noqa: E402
from paper_2105_02995_gb300.builder import build_operator  # noqa: E402
from paper_2105_02995_gb300.inputs import complex_gaussian  # noqa: E402


def test_bounded_wait_gives_up_and_device_stays_usable():
    fbuild.build()
    lib = binding.load()
    gave_up = ctypes.c_int(-1)
    rc = lib.fio_selftest_wait(20000, 8, ctypes.byref(gave_up), None)  # 20 ms limit, 8 CTAs
    assert rc == -5  # FIO_ETIMEOUT
    assert gave_up.value == 8
    buf, _ = build_operator("ex1", 256, 1e-7, 1e-6)
    op = binding.Operator(buf)
    u = complex_gaussian(256, 2, 5)
    f = op.apply_inv(binding.colmajor(torch.from_numpy(u).cuda())).cpu().numpy()
    assert np.linalg.norm(f - fa.apply_inv(fa.PackedFactors(buf), u)) / np.linalg.norm(f) < 1e-12
    assert lib.fio_selftest_wait(0, 8, ctypes.byref(gave_up), None) == -1


def test_non_convergence_is_reported():
    buf, _ = build_operator("ex1", 256, 1e-4, 1e-3)
    op = binding.Operator(buf)
    u = binding.colmajor(torch.from_numpy(complex_gaussian(256, 3, 6)).cuda())
    f, infos = op.solve(u, method=binding.FIO_GMRES, tol=1e-14, maxit=1, restart=1)
    assert all(st == -4 for _, _, st in infos)  # FIO_ENOCONV per right-hand side
    assert all(rr > 1e-14 for _, rr, _ in infos)


def test_bad_solver_options_refused():
    buf, _ = build_operator("ex1", 256, 1e-7, 1e-6)
    op = binding.Operator(buf)
    lib = binding.load()
    u = binding.colmajor(torch.from_numpy(complex_gaussian(256, 1, 7)).cuda())
    f = torch.zeros_like(u)
    opts = binding.SolveOpts(9, 0, 1e-10, 10, 10)  # no such method
    infos = (binding.SolveInfo * 1)()
    rc = lib.fio_solve(op.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(f.data_ptr()), 256, 1, 0,
                       ctypes.byref(opts), infos, None)
    assert rc == -1
