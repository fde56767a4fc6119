"""Runtime control of the BLAS thread count of the loaded OpenBLAS copies (numpy's and scipy's).

The builder runs many small LAPACK calls on a thread pool, where each call must be single
threaded, and a few large dense factorisations (the HIF root) that want every core.  OpenBLAS
exports a setter for this; this module finds the loaded OpenBLAS libraries through
/proc/self/maps and calls the setter under whichever exported name the build uses.  Where none is
found the calls are no-ops and `available()` is False.
"""

from __future__ import annotations

import contextlib
import ctypes
import os

_NAMES = ("scipy_openblas_set_num_threads64_", "scipy_openblas_set_num_threads",
          "openblas_set_num_threads64_", "openblas_set_num_threads")
_GET = ("scipy_openblas_get_num_threads64_", "scipy_openblas_get_num_threads",
        "openblas_get_num_threads64_", "openblas_get_num_threads")
_setters = None


def _find():
    global _setters
    if _setters is not None:
        return _setters
    import numpy  # noqa: F401  (load the libraries first)
    import scipy.linalg  # noqa: F401
    out = []
    try:
        with open("/proc/self/maps") as fh:
            paths = sorted({ln.split()[-1] for ln in fh if "openblas" in ln.lower() and ".so" in ln})
    except OSError:
        paths = []
    for p in paths:
        try:
            lib = ctypes.CDLL(p)
        except OSError:
            continue
        for nm in _NAMES:
            fn = getattr(lib, nm, None)
            if fn is not None:
                fn.argtypes = [ctypes.c_int]
                fn.restype = None
                get = None
                for g in _GET:
                    get = getattr(lib, g, None)
                    if get is not None:
                        get.restype = ctypes.c_int
                        break
                out.append((fn, get))
                break
    _setters = out
    return out


def available() -> bool:
    return bool(_find())


def set_threads(n: int):
    for fn, _ in _find():
        fn(int(n))


def get_threads():
    return [get() if get else None for _, get in _find()]


@contextlib.contextmanager
def threads(n: int):
    """Run the block with n BLAS threads, then restore the previous counts."""
    prev = get_threads()
    set_threads(n)
    try:
        yield
    finally:
        for (fn, _), p in zip(_find(), prev):
            if p:
                fn(p)


def pool_workers() -> int:
    """Thread-pool size for the builder: all cores when BLAS threads can be pinned to 1."""
    w = int(os.environ.get("FIO_BUILD_THREADS", os.cpu_count() or 1))
    if not available() and os.environ.get("OPENBLAS_NUM_THREADS") != "1":
        return 1  # cannot make each LAPACK call single-threaded: do not oversubscribe
    return max(1, min(32, w))
