"""Host-side logic that needs no GPU: the bench's workload naming, traffic guard and solve
summary, the serving loop's request generator, and the seeded input generator."""

import argparse
import hashlib
import os

import numpy as np

import bench
from paper_2105_02995_gb300.inputs import complex_gaussian, rhs_seed
from paper_2105_02995_gb300.serving import poisson_requests


def _args(**kw):
    base = dict(kind="ex3", n=256, b=32, eps_bf=1e-4, eps_hif=1e-3, precision="fp32")
    base.update(kw)
    return argparse.Namespace(**base)


def test_bench_names_its_workload():
    a = _args()
    assert bench.metric_of(a) == "inverse-apply RHS/s at 2D n=256"
    cfg = bench.config_of(a, {"L": 6, "LH": 4, "root": 1345}, "flushed")
    assert cfg["N"] == 65536 and cfg["b"] == 32 and "Example 3" in cfg["workload"]
    e2 = _args(kind="ex2b", n=65536, eps_bf=1e-7, eps_hif=1e-4)
    assert bench.grid_size(e2) == 65536
    assert "Example 2" in bench.config_of(e2, {}, "flushed")["workload"]
    # the arithmetic of the timed apply is named in the workload and in the config
    sp = bench.config_of(_args(precision="split_tf32"), {}, "flushed")
    assert sp["precision"] == "split_tf32" and "split-TF32" in sp["workload"]
    assert bench.PRECISIONS["split_tf32"][1] == "tf32x3"


def test_bench_traffic_guard_follows_the_kernel_source():
    """The committed traffic figure is used only while the stage-kernel source is the one the
    counters were taken from."""
    prof = os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic_ex3_n256_b32.md")
    src = os.path.join(os.path.dirname(bench.__file__), "paper_2105_02995_gb300", "csrc", "fio_kernels.cuh")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    text = open(prof).read()
    if f"kernel_source_sha256_16: {h}" in text:
        assert isinstance(bench.measured_traffic(), int) and bench.measured_traffic() > 0
    else:
        assert bench.measured_traffic() is None


def _solve(rhs, ok=True, rr=3e-11, rr64=3e-11):
    return {"statuses_ok": ok, "relres_max": rr, "relres_fp64_check": rr64, "rhs_per_s": rhs,
            "p50_ms": 1.0, "p99_ms": 1.1}


def test_bench_solve_summary_compares_at_equal_residual():
    """The summary's best mixed path is the fastest of those that converged to 1e-10 on every
    right-hand side (reported status and the FP64 recheck), and the plain path must converge."""
    solves = {"plain_fp64_pcg_b1": _solve(17.0),
              "ir_bf16_inner_dfres_b32": _solve(900.0, ok=False),              # stopped early
              "ir_tf32_inner_dfres_b32": _solve(800.0, rr64=3e-9),             # FP64 recheck fails
              "ir_split_tf32_inner_dfres_b128": _solve(240.0),
              "gmres_fp32_precond_b32": _solve(25.0),
              "error": "ignored"}
    sm = bench.solve_summary(solves)
    assert sm["best"] == "ir_split_tf32_inner_dfres_b128" and sm["rhs_per_s_ratio"] == round(240.0 / 17.0, 2)
    assert "error" in bench.solve_summary({**solves, "plain_fp64_pcg_b1": _solve(17.0, rr=2e-10)})
    assert "error" in bench.solve_summary({"plain_fp64_pcg_b1": _solve(17.0),
                                           "ir_bf16_inner_dfres_b32": _solve(900.0, ok=False)})
    assert bench.solve_converged(_solve(1.0, rr64=1.04e-10)) and not bench.solve_converged(_solve(1.0, rr64=1.06e-10))


class _Op:
    def __init__(self, N):
        self.N = N


def test_poisson_requests_are_seeded():
    ops = {"a": _Op(64), "b": _Op(256)}
    r1 = poisson_requests(ops, 20, 100.0, seed=5)
    r2 = poisson_requests(ops, 20, 100.0, seed=5)
    r3 = poisson_requests(ops, 20, 100.0, seed=6)
    assert [(r.op, r.u.shape, r.t_arrival) for r in r1] == [(r.op, r.u.shape, r.t_arrival) for r in r2]
    assert all(np.array_equal(x.u, y.u) for x, y in zip(r1, r2))
    assert [r.t_arrival for r in r1] != [r.t_arrival for r in r3]
    assert all(1 <= r.u.shape[1] <= 64 and r.u.shape[0] == ops[r.op].N for r in r1)
    assert all(np.diff([r.t_arrival for r in r1]) > 0)


def test_complex_gaussian_inputs():
    """Re and Im i.i.d. N(0, 1/2) (E|z|^2 = 1), reproducible from the seed, column-major."""
    z = complex_gaussian(4096, 8, rhs_seed(1, 2))
    assert z.dtype == np.complex128 and z.shape == (4096, 8) and z.flags.f_contiguous
    assert np.array_equal(z, complex_gaussian(4096, 8, rhs_seed(1, 2)))
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.05
    assert abs(np.mean(z.real)) < 0.05 and abs(np.mean(z.imag)) < 0.05
