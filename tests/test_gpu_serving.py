"""Batching, CUDA graphs and the serving loop on the GPU.

* A captured CUDA graph of fio_apply_inv replays to the same result as the direct call.
* The serving loop batches requests of the same operator into one launch while batches of other
  operators run on their own streams; every request's result in the mix equals its result solved
  alone, within the FP32 tolerance of the parity tests (batch widths select different kernel
  shapes, whose summation orders differ in the last bits).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2105_02995_gb300 import binding, build as fbuild  # noqa: E402
from paper_2105_02995_gb300.builder import build_operator  # noqa: E402
from paper_2105_02995_gb300.inputs import complex_gaussian  # noqa: E402
from paper_2105_02995_gb300.serving import Server, poisson_requests  # noqa: E402

TOL32 = 2e-5
_ops = {}


def ops():
    if not _ops:
        fbuild.build()
        for kind, n, eb, eh in [("ex1", 256, 1e-7, 1e-6), ("ex3", 32, 1e-5, 1e-3), ("ex1", 1024, 1e-7, 1e-6)]:
            buf, _ = build_operator(kind, n, eb, eh)
            _ops[f"{kind}_{n}"] = binding.Operator(buf)
    return _ops


@pytest.mark.parametrize("precision", [None, binding.FIO_PTF32])
def test_graph_replay_matches_direct_call(precision):
    op = ops()["ex3_32"]
    u = binding.colmajor(torch.from_numpy(complex_gaussian(op.N, 32, 17, np.complex64)).cuda())
    f = binding.colmajor(torch.empty_like(u))
    want = op.apply_inv(u, precision=precision).clone()
    g = op.capture_inv(u, f, precision)
    f.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(f, want)
    # new data in the same input buffer goes through the same graph
    u.copy_(binding.colmajor(torch.from_numpy(complex_gaussian(op.N, 32, 18, np.complex64)).cuda()))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(f, op.apply_inv(u, precision=precision))


def test_serving_results_equal_alone():
    o = ops()
    reqs = poisson_requests(o, 60, rate_per_s=20000.0, seed=4321, b_range=(1, 24))
    srv = Server(o, max_batch=64)
    srv.warmup()
    st = srv.run(reqs)
    summ = st.summary()
    assert summ["requests"] == len(reqs)
    assert st.launches < len(reqs)  # same-operator requests were batched
    assert {r.op for r in reqs} == set(o)
    for r in reqs:
        op = o[r.op]
        ud = binding.colmajor(torch.from_numpy(r.u).cuda())
        alone = op.apply_inv(ud).cpu().numpy()
        err = np.linalg.norm(r.f - alone) / np.linalg.norm(alone)
        assert err < TOL32, (r.rid, r.op, r.u.shape, err)
        assert r.t_done >= r.t_arrival


def test_serving_admission_respects_budget():
    o = ops()
    reqs = poisson_requests(o, 30, rate_per_s=50000.0, seed=99, b_range=(8, 32))
    one = max(2 * op.N * 32 * 8 for op in o.values())
    srv = Server(o, max_batch=64, hbm_budget=2 * one)
    st = srv.run(reqs)
    assert st.max_inflight_bytes <= 2 * one
    assert len(st.latencies_ms) == len(reqs)


def test_serving_solve_mode_results_equal_alone():
    """Solve requests (iterative refinement to 1e-10: double-float residuals, FP32 corrections),
    batched per operator and run by one worker thread per operator: every request converges, and
    its solution equals the same request solved alone to within what two solutions with relative
    residual <= 1e-10 can differ by on these well-conditioned operators (1e-8)."""
    o = ops()
    reqs = poisson_requests(o, 24, rate_per_s=5000.0, seed=777, b_range=(1, 12))
    srv = Server(o, max_batch=64, mode="solve")
    srv.warmup()
    st = srv.run(reqs)
    assert st.summary()["requests"] == len(reqs)
    assert st.launches < len(reqs)
    for r in reqs:
        assert r.f.dtype == np.complex128 and r.f.shape == r.u.shape
        assert all(s == 0 and rr <= 1e-10 for _, rr, s in r.info), r.info
        op = o[r.op]
        ud = binding.colmajor(torch.from_numpy(r.u.astype(np.complex128)).cuda())
        alone, infos = op.solve(ud, **srv.solve_kw)
        alone = alone.cpu().numpy()
        err = np.linalg.norm(r.f - alone) / np.linalg.norm(alone)
        assert err < 1e-8, (r.rid, r.op, r.u.shape, err)
