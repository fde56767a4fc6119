"""ctypes binding of libfio (include/fio.h): argument marshalling only.

Every computation happens in the CUDA library; this module checks shapes and dtypes, passes
pointers, sizes and the current torch stream, and turns status codes into exceptions.  It never
computes anything itself and has no CPU fallback: ``load()`` raises when libfio.so is missing.

Vectors are torch tensors on the GPU of shape (N,) or (N, b), column-major (stride (1, ld)),
complex128 (FP64 path) or complex64 (FP32 path).  ``colmajor`` makes such a tensor.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfio.so")

FIO_C128, FIO_C64 = 0, 1
FIO_P64, FIO_P32, FIO_PTF32, FIO_PBF16, FIO_PTF32X3, FIO_PDF = 0, 1, 2, 3, 4, 5
FIO_DIRECT, FIO_PCG, FIO_GMRES, FIO_IR = 0, 1, 2, 3
FIO_MASK_P64, FIO_MASK_P32, FIO_MASK_TC, FIO_MASK_DF = 1, 2, 4, 8
STATUS = {0: "FIO_OK", -1: "FIO_EINVAL", -2: "FIO_ENOMEM", -3: "FIO_EBADFACTORS",
          -4: "FIO_ENOCONV", -5: "FIO_ETIMEOUT", -6: "FIO_ECUDA", -7: "FIO_ENOTSUP"}
SYMBOLS = ["fio_upload_factors", "fio_apply_K", "fio_apply_Kadj", "fio_apply_G", "fio_apply_inv",
           "fio_apply_F", "fio_apply_Finv",
           "fio_apply_inv_host", "fio_solve", "fio_query", "fio_launch_count", "fio_apply_profiled",
           "fio_apply_inv_noalloc", "fio_selftest_wait", "fio_autotune", "fio_set_variant", "fio_stage_errors",
           "fio_sync", "fio_probe_fp32", "fio_release", "fio_strerror"]

_lib = None


class FioError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} ({_lib.fio_strerror(status).decode() if _lib else ''})")


class SolveOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("inner", ctypes.c_int), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("restart", ctypes.c_int), ("outer", ctypes.c_int),
                ("residual_op", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("relres", ctypes.c_double), ("status", ctypes.c_int)]


def load(path: str = LIB_PATH):
    """Load libfio.so (raises OSError when it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libfio.so not found at {path}; run paper_2105_02995_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.fio_upload_factors.argtypes = [vp, ctypes.c_size_t, ctypes.c_uint, vp, ctypes.POINTER(vp)]
    for name in ("fio_apply_K", "fio_apply_Kadj", "fio_apply_G", "fio_apply_inv", "fio_apply_inv_host",
                 "fio_apply_inv_noalloc", "fio_apply_F", "fio_apply_Finv"):
        getattr(lib, name).argtypes = [vp, vp, vp, i64, c_int, c_int, c_int, vp]
    lib.fio_solve.argtypes = [vp, vp, vp, i64, c_int, c_int, ctypes.POINTER(SolveOpts),
                              ctypes.POINTER(SolveInfo), vp]
    lib.fio_query.argtypes = [vp, ctypes.POINTER(c_int), ctypes.POINTER(i64), ctypes.POINTER(i64),
                              ctypes.POINTER(ctypes.c_size_t)]
    lib.fio_launch_count.argtypes = [vp, c_int, c_int, ctypes.POINTER(c_int)]
    lib.fio_apply_profiled.argtypes = [vp, c_int, vp, vp, i64, c_int, c_int, c_int, vp,
                                       ctypes.POINTER(ctypes.c_float), c_int, ctypes.POINTER(c_int)]
    lib.fio_selftest_wait.argtypes = [c_int, c_int, ctypes.POINTER(c_int), vp]
    lib.fio_autotune.argtypes = [vp, c_int, c_int, vp, ctypes.POINTER(c_int), c_int, ctypes.POINTER(c_int)]
    lib.fio_set_variant.argtypes = [vp, c_int, c_int, c_int]
    lib.fio_stage_errors.argtypes = [vp, c_int, vp, i64, c_int, c_int, vp, ctypes.POINTER(ctypes.c_double),
                                     c_int, ctypes.POINTER(c_int)]
    lib.fio_sync.argtypes = [vp]
    lib.fio_probe_fp32.argtypes = [c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(c_int), vp]
    lib.fio_release.argtypes = [vp]
    lib.fio_strerror.argtypes = [c_int]
    lib.fio_strerror.restype = ctypes.c_char_p
    for name in SYMBOLS:
        if name != "fio_strerror":
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != 0:
        raise FioError(rc, what)


def probe_fp32(iters: int = 1 << 16):
    """Measured FP32 FMA throughput of the current device (fio_probe_fp32): (TFLOP/s, ms, SMs)."""
    lib = load()
    tf, ms, sms = ctypes.c_double(), ctypes.c_float(), ctypes.c_int()
    _check(lib.fio_probe_fp32(iters, ctypes.byref(tf), ctypes.byref(ms), ctypes.byref(sms), _stream()),
           "fio_probe_fp32")
    return tf.value, ms.value, sms.value


def colmajor(t):
    """A column-major copy of a (N, b) torch tensor (or the tensor itself if it already is)."""
    if t.dim() == 1 or (t.stride(0) == 1 and t.stride(1) >= t.shape[0]):
        return t
    return t.t().contiguous().t()


def _vec(t, N):
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dtype == torch.complex128:
        dtype, prec = FIO_C128, FIO_P64
    elif t.dtype == torch.complex64:
        dtype, prec = FIO_C64, FIO_P32
    else:
        raise ValueError(f"unsupported dtype {t.dtype}")
    if t.dim() == 1:
        if t.shape[0] != N or t.stride(0) != 1:
            raise ValueError("vector must have N contiguous entries")
        return dtype, prec, 1, N
    if t.shape[0] != N or t.stride(0) != 1:
        raise ValueError("expected an N x b column-major tensor (stride (1, ld))")
    return dtype, prec, t.shape[1], max(t.stride(1), N)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Operator:
    """A packed operator uploaded to the current CUDA device (fio_upload_factors)."""

    def __init__(self, packed: bytes, precisions: int = 0):
        lib = load()
        self._lib = lib
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(packed, len(packed))
        _check(lib.fio_upload_factors(buf, len(packed), precisions, _stream(), ctypes.byref(h)),
               "fio_upload_factors")
        self.h = h
        d, n, N, nb = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        _check(lib.fio_query(h, ctypes.byref(d), ctypes.byref(n), ctypes.byref(N), ctypes.byref(nb)), "fio_query")
        self.d, self.n, self.N = d.value, n.value, N.value

    def device_bytes(self) -> int:
        nb = ctypes.c_size_t()
        _check(self._lib.fio_query(self.h, None, None, None, ctypes.byref(nb)), "fio_query")
        return nb.value

    def autotune(self, b: int, precision: int):
        """Pick every stage launch's kernel variant for b right-hand sides in `precision` by
        timing (fio_autotune); returns the chosen variant per stage launch."""
        cap = 4096
        ch = (ctypes.c_int * cap)()
        n = ctypes.c_int()
        _check(self._lib.fio_autotune(self.h, b, precision, _stream(), ch, cap, ctypes.byref(n)), "fio_autotune")
        return [ch[i] for i in range(min(n.value, cap))]

    def set_variant(self, b: int, precision: int, variant: int):
        """Pin every stage launch of (precision, bucket of b) to one kernel variant (fio_set_variant)."""
        _check(self._lib.fio_set_variant(self.h, b, precision, variant), "fio_set_variant")

    def stage_errors(self, which: str, x, precision: int):
        """Relative error of `precision` against the FP64 path after every stage of the apply
        `which` (fio_stage_errors); x: complex128 column-major device tensor."""
        k = {"K": 0, "Kadj": 1, "G": 2, "inv": 3}[which]
        dt, prec, b, ld = _vec(x, self.N)
        if dt != FIO_C128:
            raise ValueError("fio_stage_errors takes complex128 input")
        cap = 4096
        out = (ctypes.c_double * cap)()
        n = ctypes.c_int()
        _check(self._lib.fio_stage_errors(self.h, k, ctypes.c_void_p(x.data_ptr()), ld, b, precision, _stream(),
                                          out, cap, ctypes.byref(n)), "fio_stage_errors")
        return [out[i] for i in range(min(n.value, cap))]

    def launches(self, which: str, b: int) -> int:
        k = {"K": 0, "Kadj": 1, "G": 2, "inv": 3}[which]
        out = ctypes.c_int()
        _check(self._lib.fio_launch_count(self.h, k, b, ctypes.byref(out)), "fio_launch_count")
        return out.value

    def _apply(self, fn, name, x, y, precision=None):
        import torch
        if y is None:
            y = torch.empty_like(colmajor(x) if x.dim() == 2 else x)
            y = colmajor(y) if y.dim() == 2 else y
        dt, prec, b, ld = _vec(x, self.N)
        dty, precy, by, ldy = _vec(y, self.N)
        if (dt, b) != (dty, by) or ld != ldy:
            raise ValueError("x and y must have the same dtype, shape and leading dimension")
        if precision is not None:
            prec = precision
        _check(fn(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), ld, b, dt,
                  prec, _stream()), name)
        return y

    def apply_profiled(self, which: str, x, y, precision=None):
        """Per-launch-group times (ms) of one apply, in launch order (fio_apply_profiled)."""
        k = {"K": 0, "Kadj": 1, "G": 2, "inv": 3}[which]
        dt, prec, b, ld = _vec(x, self.N)
        if precision is not None:
            prec = precision
        cap = 4096
        ms = (ctypes.c_float * cap)()
        nm = ctypes.c_int()
        _check(self._lib.fio_apply_profiled(self.h, k, ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(y.data_ptr()), ld, b, dt, prec, _stream(),
                                            ms, cap, ctypes.byref(nm)), "fio_apply_profiled")
        return [ms[i] for i in range(nm.value)]

    def apply_K(self, x, y=None, precision=None):
        return self._apply(self._lib.fio_apply_K, "fio_apply_K", x, y, precision)

    def apply_Kadj(self, x, y=None, precision=None):
        return self._apply(self._lib.fio_apply_Kadj, "fio_apply_Kadj", x, y, precision)

    def apply_G(self, x, y=None, precision=None):
        return self._apply(self._lib.fio_apply_G, "fio_apply_G", x, y, precision)

    def apply_F(self, f, fhat=None):
        """f-hat = F f, the DFT of section 1 (fio_apply_F)."""
        return self._apply(self._lib.fio_apply_F, "fio_apply_F", f, fhat)

    def apply_Finv(self, fhat, f=None):
        """f = F^{-1} f-hat (fio_apply_Finv): with apply_inv, the full solve of u = K F f."""
        return self._apply(self._lib.fio_apply_Finv, "fio_apply_Finv", fhat, f)

    def apply_inv(self, u, f=None, precision=None):
        """f = G-dot K-dot* u; precision defaults to the dtype's (P64 / P32), or FIO_PTF32 /
        FIO_PBF16 / FIO_PTF32X3 for the tensor-core stage products on complex64 vectors."""
        return self._apply(self._lib.fio_apply_inv, "fio_apply_inv", u, f, precision)

    def capture_inv(self, u, f, precision=None):
        """A CUDA graph of one fio_apply_inv(u -> f) on these buffers; replay it with .replay().

        A first call on a side stream sizes the operator's scratch pool, so the captured call
        neither allocates nor synchronises (both are illegal while a stream is being captured)."""
        import torch
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.apply_inv(u, f, precision)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.apply_inv(u, f, precision)
        return g

    def apply_inv_host(self, u: np.ndarray, f: np.ndarray | None = None, precision=None) -> np.ndarray:
        """Host-buffer direct solve: numpy (N, b) Fortran-ordered complex128/complex64 arrays;
        precision defaults to the dtype's (P64 / P32)."""
        u = np.asfortranarray(u)
        if u.ndim == 1:
            u = u[:, None]
        if f is None:
            f = np.empty_like(u, order="F")
        if u.dtype == np.complex128:
            dt, prec = FIO_C128, FIO_P64
        elif u.dtype == np.complex64:
            dt, prec = FIO_C64, FIO_P32
        else:
            raise ValueError("complex128 or complex64 expected")
        if u.shape[0] != self.N or f.shape != u.shape or f.dtype != u.dtype or not f.flags.f_contiguous:
            raise ValueError("bad host arrays")
        if precision is not None:
            prec = precision
        _check(self._lib.fio_apply_inv_host(self.h, u.ctypes.data_as(ctypes.c_void_p),
                                            f.ctypes.data_as(ctypes.c_void_p), self.N, u.shape[1],
                                            dt, prec, _stream()), "fio_apply_inv_host")
        return f

    def solve(self, u, f=None, method: int = FIO_GMRES, inner: int = FIO_P64, tol: float = 1e-10,
              maxit: int = 100, restart: int = 20, outer: int = FIO_P64, residual_op=None):
        """Iterative solve of K-dot f = u (complex128 tensors); returns (f, list of (iters, relres, status)).
        outer = FIO_PDF computes the true residuals in double-float arithmetic; residual_op (an
        Operator of the same grid with a tighter butterfly; FIO_IR and FIO_DIRECT) takes them
        with that operator's K-dot instead."""
        import torch
        if f is None:
            f = torch.zeros_like(u)
        dt, prec, b, ld = _vec(u, self.N)
        if dt != FIO_C128:
            raise ValueError("fio_solve takes complex128 vectors")
        opts = SolveOpts(method, inner, tol, maxit, restart, outer,
                         residual_op.h.value if residual_op is not None else None)
        infos = (SolveInfo * max(b, 1))()
        rc = self._lib.fio_solve(self.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                 ld, b, dt, ctypes.byref(opts), infos, _stream())
        if rc not in (0, -4):
            _check(rc, "fio_solve")
        return f, [(infos[j].iters, infos[j].relres, infos[j].status) for j in range(b)]

    def sync(self):
        """Synchronise the current stream; raises FioError(FIO_ETIMEOUT) when a tensor-core
        bounded wait gave up in an earlier asynchronous apply (fio_sync)."""
        _check(self._lib.fio_sync(_stream()), "fio_sync")

    def release(self):
        if getattr(self, "h", None):
            self._lib.fio_release(self.h)
            self.h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class NormalMatvecGPU:
    """K-dot* K-dot X on the GPU for the builder's peeling probes (bind() takes the butterfly
    stages and uploads them as a butterfly-only operator)."""

    def __init__(self, precision: int = FIO_P64, chunk: int = 256):
        self.precision = precision
        self.chunk = chunk

    def bind(self, bf_stages, d: int, n: int):
        from .builder.pack import pack
        packed = pack(d, n, bf_stages, [], [], 0.0, 0.0)
        op = Operator(packed)
        prec = self.precision
        chunk = self.chunk

        def mv(X):
            import torch
            X = np.asarray(X)
            out = np.empty((X.shape[0], X.shape[1]), dtype=np.complex128)
            dt = torch.complex128 if prec == FIO_P64 else torch.complex64
            for s in range(0, X.shape[1], chunk):
                xb = torch.from_numpy(np.ascontiguousarray(X[:, s:s + chunk].T)).to("cuda", dt).t()
                yb = op.apply_K(xb)
                zb = op.apply_Kadj(yb)
                out[:, s:s + chunk] = zb.t().cpu().numpy().T
            return out

        mv.op = op
        return mv
