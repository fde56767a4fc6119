"""Full-size GPU checks at the workload sizes, against the oracle's definition of K.

At these sizes the dense oracle does not fit, so the checks use what the oracle computes one by
one (oracle/fio_oracle.py): sampled rows of K f and sampled columns of K (hence entries of K* u),
O(N) each.  Checked:
  * K-dot and K-dot* against K at sampled outputs: relative error within a small multiple of the
    butterfly tolerance (the paper's e_a is of the order of eps_BF);
  * the direct solve f = G-dot K-dot* u: sampled residual (K f - u)_S / ||u_S|| within the order
    of the paper's e_s at these sizes (Tables for Examples 1 and 3);
  * GMRES / PCG to 1e-10 on K-dot f = u: iteration counts of the order the paper reports with G
    as preconditioner, and the sampled residual against the true K within e_a.
And against the oracle's FP64 product of the same packed factors (oracle/factor_apply.py), at
the benchmark's configuration (2D n = 256, complex64, 32 right-hand sides, autotuned kernels) and
at 1D N = 16384 with eps = 1e-9 (the tight-tolerance Example 1 operator), element-wise.
Operators are built once per box and cached on disk (shared with bench.py).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fio_oracle as fo  # noqa: E402
from paper_2105_02995_gb300 import binding, build as fbuild  # noqa: E402
from paper_2105_02995_gb300.builder.__main__ import build_cached  # noqa: E402
from paper_2105_02995_gb300.inputs import complex_gaussian, rhs_seed  # noqa: E402

CASES = {
    # kind, n, eps_bf, eps_hif, dtype, K bound, direct-solve bound: about three times the values
    # measured on a GB300 with these seeds (K-dot / K-dot* at sampled outputs; direct solve):
    #   ex1_65536     2.1e-7 / 5.6e-8;   3.9e-7
    #   ex3_256       3.0e-4 / 5.2e-4;   1.9e-3
    #   ex1_16384_e9  1.3e-10 / 4.6e-11; 3.9e-10 (the same on the host with the oracle)
    "ex1_65536": ("ex1", 65536, 1e-7, 1e-6, torch.complex128, 7e-7, 1.2e-6),
    "ex3_256": ("ex3", 256, 1e-4, 1e-3, torch.complex64, 1.6e-3, 6e-3),
    "ex1_16384_e9": ("ex1", 16384, 1e-10, 1e-9, torch.complex128, 4e-10, 1.2e-9),
}
TOL64, TOL32 = 1e-12, 2e-5  # as in tests/test_gpu_parity.py
_ops = {}
_packed = {}


def get(name):
    if name not in _ops:
        fbuild.build()
        kind, n, eb, eh, dt, kb, sb = CASES[name]
        buf, info = build_cached(kind, n, eb, eh, gpu=True, verbose=False)
        _ops[name] = (binding.Operator(buf), fo.FIO(kind, n), info)
        _packed[name] = buf
    return _ops[name]


def factors(name):
    """The oracle's parse of the packed factors (sparse FP64 stage matrices)."""
    from oracle import factor_apply as fa
    get(name)
    key = name + "/parsed"
    if key not in _packed:
        _packed[key] = fa.PackedFactors(_packed[name], verify=False)
    return _packed[key]


def dev(a, dtype):
    return binding.colmajor(torch.from_numpy(np.asarray(a)).to("cuda", dtype))


def rel(a, b):
    """Frobenius ratio: the norm of the paper's error measures e_a, e_s."""
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def relmax(a, b):
    """Parity measure: max(||a - b||_F / ||b||_F, max|a - b| / max|b|)."""
    return max(rel(a, b), float(np.abs(a - b).max() / np.abs(b).max()))


@pytest.mark.parametrize("name", list(CASES))
def test_butterfly_at_sampled_outputs(name):
    op, ofo, info = get(name)
    kind, n, eb, eh, dt, kbound, _ = CASES[name]
    N, b = ofo.N, 2
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(N, 48, replace=False))
    f = complex_gaussian(N, b, rhs_seed(3))
    u = op.apply_K(dev(f, dt)).cpu().numpy().astype(np.complex128)
    want = fo.K_rows(ofo, rows, f.astype(np.complex64).astype(np.complex128) if dt == torch.complex64 else f)
    print(f"[{name}] K-dot vs K at sampled rows: {rel(u[rows], want):.3g}")
    assert rel(u[rows], want) < kbound
    # K* x at sampled outputs: (K* x)_j = sum_i conj(K_ij) x_i, one column of K at a time
    x = complex_gaussian(N, b, rhs_seed(3, 1))
    y = op.apply_Kadj(dev(x, dt)).cpu().numpy().astype(np.complex128)
    cols = rows[:16]
    Kc = fo.K_block(ofo, np.arange(N), cols)
    xx = x.astype(np.complex64).astype(np.complex128) if dt == torch.complex64 else x
    print(f"[{name}] K-dot* vs K* at sampled outputs: {rel(y[cols], Kc.conj().T @ xx):.3g}")
    assert rel(y[cols], Kc.conj().T @ xx) < kbound


@pytest.mark.parametrize("name", list(CASES))
def test_direct_solve_sampled_residual(name):
    op, ofo, info = get(name)
    kind, n, eb, eh, dt, kbound, sbound = CASES[name]
    N, b = ofo.N, 4
    u = complex_gaussian(N, b, rhs_seed(4))
    f = op.apply_inv(dev(u, dt)).cpu().numpy().astype(np.complex128)
    rows = np.sort(np.random.default_rng(5).choice(N, 48, replace=False))
    print(f"[{name}] direct solve, sampled residual: {rel(fo.K_rows(ofo, rows, f), u[rows]):.3g}")
    assert rel(fo.K_rows(ofo, rows, f), u[rows]) < sbound


@pytest.mark.parametrize("name,method", [("ex1_65536", binding.FIO_PCG), ("ex1_65536", binding.FIO_GMRES),
                                         ("ex3_256", binding.FIO_GMRES), ("ex3_256", binding.FIO_IR),
                                         ("ex1_16384_e9", binding.FIO_GMRES)])
def test_iterative_solve_full_size(name, method):
    op, ofo, info = get(name)
    kind, n, eb, eh, dt, kbound, _ = CASES[name]
    N, b = ofo.N, 2
    u = complex_gaussian(N, b, rhs_seed(5))
    inner = binding.FIO_P32 if dt == torch.complex64 else binding.FIO_P64
    f, infos = op.solve(dev(u, torch.complex128), method=method, inner=inner, tol=1e-10, maxit=60)
    for it, rr, st in infos:
        assert st == 0 and rr <= 1e-10, infos
        assert it <= 30, infos
    fh = f.cpu().numpy()
    rows = np.sort(np.random.default_rng(6).choice(N, 48, replace=False))
    res = rel(fo.K_rows(ofo, rows, fh), u[rows])
    print(f"[{name}] iterative solve ({method}), sampled residual against K: {res:.3g}")
    assert res < 20 * kbound


def test_headline_config_vs_factor_oracle():
    """The benchmark's configuration -- 2D generalized Radon transform n = 256, complex64 vectors,
    32 right-hand sides, FP32 arithmetic, every stage launch's kernel picked by the autotuner --
    against the oracle's FP64 product of the same factors on 4 of the 32 columns (the oracle
    takes ~1.5 s per column here), within the FP32 parity bound; and the FP64 path (b = 5, the
    tiled kernels) on all 5 columns within 1e-12."""
    from oracle import factor_apply as fa
    op, ofo, info = get("ex3_256")
    P = factors("ex3_256")
    N, b = ofo.N, 32
    u = complex_gaussian(N, b, rhs_seed(2))
    op.autotune(b, binding.FIO_P32)
    f = op.apply_inv(dev(u, torch.complex64)).cpu().numpy().astype(np.complex128)
    cols = [0, 9, 22, 31]
    u32 = u.astype(np.complex64).astype(np.complex128)
    want = fa.apply_inv(P, u32[:, cols])
    assert relmax(f[:, cols], want) < TOL32
    u5 = u[:, :5]
    f64 = op.apply_inv(dev(u5, torch.complex128)).cpu().numpy()
    assert relmax(f64, fa.apply_inv(P, u5)) < TOL64


@pytest.mark.parametrize("b", [1, 8, 64])
def test_ex1_tight_tolerance_vs_factor_oracle(b):
    """Example 1 at N = 16384 with eps = 1e-9 (eps_BF = 1e-10), complex128: K-dot, K-dot* and
    G-dot K-dot* against the oracle's FP64 product of the same factors within 1e-12, at the
    right-hand-side counts 1, 8 and 64."""
    from oracle import factor_apply as fa
    op, ofo, info = get("ex1_16384_e9")
    P = factors("ex1_16384_e9")
    x = complex_gaussian(ofo.N, b, rhs_seed(1, b))
    xd = dev(x, torch.complex128)
    for what, ref in (("K", fa.apply_Kdot), ("Kadj", fa.apply_Kdot_adj), ("inv", fa.apply_inv)):
        y = getattr(op, "apply_" + what)(xd).cpu().numpy()
        assert relmax(y, ref(P, x)) < TOL64, (what, b)
